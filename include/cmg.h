/*
 * cmg.h -- C ABI of the GB300 compact full multigrid (CMG) library.
 *
 * The library solves -Lap u = f with zero Dirichlet data on the unit square
 * (d = 2) or cube (d = 3), P1 elements on the structured Kuhn triangulation,
 * by compact FMG with iterative refinement (Algorithm 3 of "Multigrid with
 * Linear Storage Complexity", Bauer, Kohl, McCormick, Tamstorf).  The solution
 * u~, the residual r and the correction y~ live in the compact representation
 * (Sec. 2, eq. compact-to-standard): one block-floating-point (BFP) section per
 * grid level, widths regressive in the level (Table 1, eq. regressive).
 *
 * Conventions
 *  - Every call returns a cmg_status; nothing aborts or throws across the ABI.
 *    CUDA failures map to CMG_ECUDA, with the text in cmg_last_error().
 *  - Work is enqueued on the CUDA stream given at creation (or per call for the
 *    stand-alone codec).  Calls marked "synchronises" wait for that stream.
 *  - Device pointers ("_dev") may come from any allocator (e.g. torch); the
 *    library never frees memory it did not allocate.  Host pointers ("_host")
 *    are read or written before the call returns.
 *  - Levels: level l has 2^l - 1 interior nodes per axis (h = 2^-l); level 1 is
 *    the coarsest (one unknown).  Dense level arrays are x-fastest, then y, z.
 *
 * BFP layout (bit-exact contract).  A section on level l stores each x-row of
 * 2^l - 1 values as ceil((2^l - 1)/32) blocks of 32 (zero padded).  A block has
 * one int8 exponent e and W uint32 words holding 32 W-bit two's-complement codes
 * q_i (2 <= W <= 32, sign bit included): value_i = q_i * 2^(e-W+1); code i sits
 * at bits [iW, iW+W) of the block's little-endian word stream.  e is the
 * smallest integer with max|x| < 2^e, codes are rounded to nearest with ties to
 * even (Sec. 4), and the exponent is raised by one when a code would reach
 * 2^(W-1).  An all-zero block stores e = -128.  Blocks are ordered by row
 * (x-block fastest, then y, then z); words are stored block after block.
 */
#ifndef CMG_H
#define CMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CMG_OK = 0,
  CMG_EINVAL = 1,       /* bad argument or parameter combination */
  CMG_ENOMEM = 2,       /* device or host allocation failed */
  CMG_ERANGE = 3,       /* exponent outside [-127, 127], or the exact integer
                           arithmetic would need more than 62 bits */
  CMG_ECUDA = 4,        /* CUDA runtime error (see cmg_last_error) */
  CMG_ECORRUPT = 5,     /* code -2^(W-1) met while decoding */
  CMG_ETIMEOUT = 6,     /* reserved: no call waits on a device flag */
  CMG_EUNSUPPORTED = 7  /* a valid request the library does not implement */
} cmg_status;

/* Parameters of Algorithm 3 with the precisions of Table 1 (P1: p = 1, m = 1).
 * Intermediate arithmetic is exact (fixed-point integers on the GPU); values are
 * rounded only where they are stored, as the paper's rounding rules prescribe. */
enum { CMG_ARITH_EXACT = 0, CMG_ARITH_FP32 = 1, CMG_ARITH_FP64 = 2 };
enum { CMG_COEF_POISSON = 0, CMG_COEF_DIFFUSION = 1 };
enum { CMG_SMOOTHER_JACOBI = 0, CMG_SMOOTHER_RBGS = 1 };

typedef struct {
  int dim;             /* 2 or 3 */
  int L_max;           /* finest level, 1 <= L_max <= 14 (3-D: <= 12, so that
                          the finest level has fewer than 2^31 BFP blocks) */
  int b1;              /* finest-level width of u~ (Table 1 b_1), 2..32 */
  int b2;              /* finest-level width of r and y~ (Table 1 b_2), 2..32 */
  int k_u;             /* regressive increment of u~, p + 1 = 2 */
  int k_r;             /* regressive increment of r and y~, m = 1 */
  int N_ir;            /* IR iterations per FMG level (Algorithm 3 N) */
  int nu1, nu2;        /* pre-/post-smoothing sweeps, nu1 >= 0, nu2 >= 1 */
  int omega_num;       /* Jacobi weight omega = omega_num / 2^omega_log2den, */
  int omega_log2den;   /* which must make omega / (2d) a dyadic rational */
  int arith;           /* CMG_ARITH_EXACT (0): exact V-cycle; CMG_ARITH_FP32 (1):
                          the V-cycle (sweeps, inner residuals, restriction input,
                          prolongated corrections) in binary32, round to nearest,
                          in a fixed order, inside the exact iterative refinement
                          (outer residual, level-1 solve and u~ correction exact);
                          needs k_r (L_max - 1) + b2 + bitlen(Jacobi numerator) <= 24;
                          CMG_ARITH_FP64 (2): the same cycle in binary64, the plain
                          FP64 form of the precision split of Table 1 */
  int coef;            /* CMG_COEF_POISSON (0): -Lap u = f; CMG_COEF_DIFFUSION (1):
                          -div(k grad u) = f with the nodal coefficient set by
                          cmg_set_coefficient; needs arith = CMG_ARITH_FP32 or
                          CMG_ARITH_FP64 and nu1 >= 1 (the outer residual and
                          level-1 solve in FP64, the cycle in binary32 or binary64,
                          each in a fixed order) */
  int smoother;        /* CMG_SMOOTHER_JACOBI (0): weighted Jacobi sweeps;
                          CMG_SMOOTHER_RBGS (1): red-black Gauss-Seidel post-
                          smoothing (Algorithm 1 as the V(0,1) cycle of Sec. 7):
                          each of the nu2 sweeps updates the red nodes (the sum
                          of the 1-based node numbers even), then the black ones,
                          each half-sweep with the damped point update
                          y <- y + omega/(2d) h^(2-d) (rc - A(y + z)) and rounded
                          into the BFP section; needs nu1 = 0 and coef = 0 */
} cmg_params;

/* Per-solve report filled by cmg_fmg_solve. */
typedef struct {
  double solve_ms;        /* device time of the whole FMG (CUDA events) */
  int64_t dofs;           /* interior unknowns on the finest level */
  int64_t launches;       /* launch steps of the solve: one per kernel, except
                             that a restriction step of a diffusion problem
                             (coef = 1) runs two kernels and counts once */
  double alg_bytes;       /* algorithmic bytes moved by all kernels (model):
                             sections, exponents and temporaries; the reads
                             of a diffusion problem's coefficient field are
                             not included */
  double persistent_bits; /* compact u~, r, y~ (x2) storage at L_max, all levels,
                             mantissas + exponents + padding */
  double temp_bytes;      /* int64 temporaries (levels <= L_max-1) and, with
                             nu1 = 0, the restriction chain's t^ sections
                             ((p+1) L_max + b1 bits, levels <= L_max-1) */
  /* dominant kernel statistics (finest-level sweeps and residuals, bytes as
   * alg_bytes); the times are valid when timing is enabled (cmg_set_timing). */
  double sweep_ms_total;
  int64_t sweep_launches;
  double sweep_alg_bytes;
  double resid_ms_total;
  int64_t resid_launches;
  double resid_alg_bytes;
} cmg_report;

/* Kernel kinds for cmg_kernel_stats. */
enum {
  CMG_KIND_RESIDUAL = 0,   /* fmgResidual (Algorithm 2), first sweep fused */
  CMG_KIND_SWEEP = 1,      /* Jacobi sweeps, corrections fused */
  CMG_KIND_RESTRICT = 2,   /* restriction into the int64 accumulator */
  CMG_KIND_ACC_ENCODE = 3, /* accumulator to BFP (restricted right-hand side) */
  CMG_KIND_COARSE = 4,     /* level-1 solve */
  CMG_KIND_REPACK = 5,     /* FMG level step (widening) */
  CMG_KIND_OTHER = 6,      /* decode chain and step-wise pieces */
  CMG_KIND_COUNT = 7
};

/* Section selectors for cmg_get_section / cmg_set_section. */
enum { CMG_SEC_U = 0, CMG_SEC_R = 1, CMG_SEC_RC = 2, CMG_SEC_Y = 3 };

typedef struct cmg_ctx cmg_ctx;

/* ---------------------------------------------------------------------------
 * Stand-alone BFP codec (Sec. 6.1.3).  n values, blocks of 32 consecutive
 * values (the last one zero padded).  words_dev: ceil(n/32)*W uint32,
 * exps_dev: ceil(n/32) int8, all device memory owned by the caller.
 * encode: CMG_EINVAL for W outside 2..32 or a non-finite input, CMG_ERANGE for
 * an exponent outside [-127, 127].  decode: CMG_ECORRUPT for a code -2^(W-1)
 * (the value is then written as if the code were valid).  Both synchronise
 * the given stream to report data-dependent errors. */
cmg_status cmg_encode(const double *x_dev, int64_t n, int W, uint32_t *words_dev,
                      int8_t *exps_dev, void *cuda_stream);
cmg_status cmg_decode(const uint32_t *words_dev, const int8_t *exps_dev, int64_t n, int W,
                      double *x_dev, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Solver context: allocates the compact hierarchy for L_max (device memory it
 * owns) and binds a CUDA stream (NULL = default stream).  Validation only,
 * no device work: cmg_params_check. */
cmg_status cmg_params_check(const cmg_params *p);
cmg_status cmg_create(const cmg_params *p, void *cuda_stream, cmg_ctx **out);
void cmg_destroy(cmg_ctx *ctx);
const char *cmg_last_error(const cmg_ctx *ctx); /* never NULL */
/* Per-launch CUDA events on the context's stream, read by cmg_kernel_stats and
 * the report: mode 0 none (the default), 1 around every launch, 2 around the
 * launches on level L_max only (the dominant kernels; the events add a few
 * microseconds per launch, which matters for small hierarchies).  CMG_EINVAL
 * for another mode. */
cmg_status cmg_set_timing(cmg_ctx *ctx, int mode);
/* Specialised kernels (3-D exact path; on by default): the red half-sweep from
 * y~ = 0, the black half-sweep with the correction of u~ and the residual with
 * the restriction of t^_L run in kernels with 32-bit arithmetic where per-CTA
 * and per-block bounds allow it (other tiles and blocks run exactly in 64 bits).
 * They compute the same bits as the generic kernels; enable = 0 runs the
 * generic kernels only (for comparisons).  Takes effect at the next launch. */
cmg_status cmg_set_fast_kernels(cmg_ctx *ctx, int enable);
/* CTAs (32 x 8 x 32-node tiles) the specialised kernels were launched with since
 * the last cmg_start (or the solve's start), and how many of them left their
 * tile to the generic kernel because the tile's footprint exceeds the kernel's
 * number range; top = 1 counts only launches on level L_max.  Synchronises. */
cmg_status cmg_fast_stats(cmg_ctx *ctx, int top, int64_t *ctas, int64_t *fallback_ctas);
/* Two-level coarse sources (exact Poisson path with L_max >= 3): on the finest
 * FMG level the sweeps, the residual and the decode form w_(L-1) and
 * u^_(L-1) from the level-(L-1) section (y~ or u~) and the level-(L-2) int64
 * temporary when a tile stages them (Sec. 6.1: only the compact sections are
 * kept per level), so that level L_max - 1 holds no int64 copy of them
 * (enable = 1 frees those two arrays, 16 bytes per level-(L_max - 1) node;
 * enable = 0 allocates them again and reads them materialized).  Both give the
 * same bits; off by default (the materialized sources take fewer instructions
 * per value).  Synchronises the stream; call it between solves.  EUNSUPPORTED
 * for other configurations (enable = 0 is then a no-op). */
cmg_status cmg_set_two_level(cmg_ctx *ctx, int enable);
/* The solve as one CUDA graph (on by default).  The host logic of cmg_fmg_solve
 * depends only on the context's inputs and configuration, never on device
 * data: after one eager solve of the current inputs, the next solve captures
 * its whole launch sequence (kernels, memsets and, with timing, the event
 * records) into a graph and launches it, and later solves launch that graph
 * again, with the same kernels, arguments and results.  Any call that changes
 * an input or the configuration drops the graph: the setters of timing, the
 * specialised kernels and the two-level sources when they change the setting,
 * cmg_set_rhs_separable unless the tables and scale are the same as before,
 * cmg_set_coefficient / cmg_set_rhs_nodal when the pointer or scale changes
 * (the graph reads borrowed arrays through their pointers, so new contents at
 * the same address need no new graph), the step calls, cmg_set_section and
 * cmg_state_load.  Not used on the legacy default stream (NULL), which cannot
 * be captured; a capture that fails solves eagerly.  enable = 0 drops the
 * graph and solves eagerly. */
cmg_status cmg_set_graphs(cmg_ctx *ctx, int enable);
/* Graphs captured, and solves run as a launch of the solve's graph (the
 * capturing solve included), since cmg_create. */
cmg_status cmg_graph_stats(const cmg_ctx *ctx, int64_t *captures, int64_t *graph_solves);

/* Right-hand side (matrix-free, Sec. 5.1): F(x) = 2^scale_exp * sum_t prod_a
 * T[t][a][i_a], with T an int32 table [nterms][dim][2^L_max - 1] sampled at the
 * finest interior nodes (copied; the caller keeps ownership).  The nodal load
 * f_L = h_L^d F is rounded to nearest-even on the grid 50 bits below the bound
 * sum_t prod_a max|T[t][a]|.  |T| must be <= 2^30 and nterms <= 64. */
cmg_status cmg_set_rhs_separable(cmg_ctx *ctx, int nterms, const int32_t *tables_host,
                                 int scale_exp);

/* Diffusion: the nodal coefficient k on the finest grid, boundary nodes
 * included, (2^L_max + 1)^dim binary32 values, x fastest, in device memory the
 * caller keeps alive and unchanged while the context uses it (borrowed; n must
 * equal that count).  Level l reads it at stride 2^(L_max - l) (injection); the
 * flux between neighbours uses the face value (k_p + k_q) / 2. */
cmg_status cmg_set_coefficient(cmg_ctx *ctx, const float *k_dev, int64_t n);

/* Diffusion: a right-hand side given by nodal values g at the interior nodes
 * of the finest grid ((2^L_max - 1)^dim doubles in device memory, borrowed
 * like the coefficient): f_L = h_L^d 2^scale_log2 g, injected at stride
 * 2^(L_max - L) on coarser FMG levels (the power-of-two scale is exact unless
 * a value leaves the binary64 range).  Replaces cmg_set_rhs_separable (used by
 * adjoint solves, whose right-hand side du J is not separable: A lam = du J is
 * posed with g = du J and scale_log2 = d L_max, since A lam = h^d g' needs
 * g' = 2^(d L_max) du J).  CMG_EINVAL for |scale_log2| > 512. */
cmg_status cmg_set_rhs_nodal(cmg_ctx *ctx, const double *g_dev, int64_t n, int scale_log2);

/* Adjoint gradients of J(u) for -div(k grad u) = g with A u = h^d g and the
 * adjoint state lam solving A lam = dJ/du (A is symmetric), on device arrays:
 *   dk_dev[i] = dJ/dk_i = -(1/2) h^(d-2) sum over the neighbours q of node i in
 *               the closed finest grid (order -x,+x,-y,+y,-z,+z) of
 *               (u_i - u_q)(lam_i - lam_q), every node, boundary included
 *               ((2^L_max + 1)^dim doubles; u = lam = 0 on the boundary);
 *   dg_dev[p] = dJ/dg_p = h^d lam_p on the interior (may be NULL).
 * u and lam are interior arrays ((2^L_max - 1)^dim doubles), x fastest.  FP64 in
 * that fixed order.  Enqueued on the context's stream. */
cmg_status cmg_gradient(cmg_ctx *ctx, const double *u_dev, const double *lam_dev, double *dk_dev,
                        double *dg_dev);

/* Algorithm 3 end to end (coarse solve, then L = 2..L_max with N_ir IR
 * iterations each).  Synchronises; fills *report when non-NULL. */
cmg_status cmg_fmg_solve(cmg_ctx *ctx, cmg_report *report);

/* Launch statistics of the last cmg_fmg_solve per kernel kind (CMG_KIND_*),
 * for launches on level L_max (top = 1) or on coarser levels (top = 0): total
 * device time (CUDA events on the context's stream; 0 for launches that
 * cmg_set_timing leaves without events), number of launches and modelled
 * algorithmic bytes. */
cmg_status cmg_kernel_stats(cmg_ctx *ctx, int kind, int top, double *ms, int64_t *launches,
                            double *bytes);

/* Individual steps of Algorithm 3 (unfused kernels), for step-wise checking.
 * cmg_start: L = 1, u~_1 = round(f_1 / A_1).  cmg_prolongate: FMG level step
 * (zero new section, widen the coarser ones by k_u bits).  cmg_residual:
 * Algorithm 2 at the current level.  cmg_down(l): nu1 sweeps on level l from
 * y~ = 0 and the restriction rc_(l-1) = round(R_l (rc_l - A_l y~_l)).
 * cmg_coarse: y~_1 = round(rc_1 / A_1).  cmg_up(l): nu2 sweeps on level l with
 * z_l = P_l w_(l-1), then w_l = y~_l + z_l.  cmg_correct: u~_l += y~_l (all l).
 * cmg_vcycle: the down legs, coarse solve and up legs.  cmg_ir_iteration: one
 * residual + cycle + correction with the fused production kernels.
 * cmg_smooth(l, sweeps, with_z): the smoothing of Algorithm 1 on level l
 * (2 <= l <= L): with_z = 0 runs `sweeps` pre-smoothing sweeps from y~_l = 0
 * (Jacobi only, CMG_EUNSUPPORTED with red-black Gauss-Seidel); with_z = 1 runs
 * `sweeps` post-smoothing sweeps on eq. cfas with z_l = P_l w_(l-1) (needs
 * w_(l-1): cmg_coarse or cmg_up on level l-1 first), the last one writing
 * w_l = y~_l + z_l.  cmg_restrict(l): rc_(l-1) = round(R_l (rc_l - A_l y~_l));
 * CMG_EUNSUPPORTED without pre-smoothing, where the residual's restriction
 * chain forms every rc_l (Algorithm 2).  cmg_down(l) is cmg_smooth(l, nu1, 0)
 * then cmg_restrict(l); cmg_up(l) is cmg_smooth(l, nu2, 1).
 * Errors: CMG_EINVAL for a NULL context, a level outside 2..L (L = cmg_level),
 * or a call before cmg_start; CMG_EUNSUPPORTED for a cycle on a one-level
 * hierarchy; data-dependent errors (CMG_ERANGE, CMG_ECORRUPT) surface at the
 * next synchronising call (cmg_sync). */
cmg_status cmg_start(cmg_ctx *ctx);
cmg_status cmg_prolongate(cmg_ctx *ctx);
cmg_status cmg_residual(cmg_ctx *ctx);
cmg_status cmg_down(cmg_ctx *ctx, int level);
cmg_status cmg_coarse(cmg_ctx *ctx);
cmg_status cmg_up(cmg_ctx *ctx, int level);
cmg_status cmg_smooth(cmg_ctx *ctx, int level, int sweeps, int with_z);
cmg_status cmg_restrict(cmg_ctx *ctx, int level);
cmg_status cmg_correct(cmg_ctx *ctx);
cmg_status cmg_vcycle(cmg_ctx *ctx);
cmg_status cmg_ir_iteration(cmg_ctx *ctx);
int cmg_level(const cmg_ctx *ctx); /* current FMG level L (0 before cmg_start) */
/* Waits for the stream and reports data-dependent errors (CMG_ERANGE, ...). */
cmg_status cmg_sync(cmg_ctx *ctx);

/* Section access (synchronises).  which: CMG_SEC_*; level 1..L.  words_host:
 * nblocks * W uint32 where W is cmg_section_width(); exps_host: nblocks int8;
 * both host memory of the caller, written before the call returns
 * (cmg_get_section takes words_host = NULL to read the exponents only).
 * cmg_get_section writes page-locked host memory (cudaHostAlloc,
 * cudaHostRegister) that is 16-byte aligned with a copy kernel on the
 * context's stream, through the GPU's mapping of the buffer (both ends of the
 * range must be mapped), and other host memory with cudaMemcpy; the buffer
 * must hold the sizes above either way.
 * cmg_set_section copies a caller's section in (for checkpoint restore and
 * step-wise checking); W must lie in 2..32 and not exceed the width the section
 * was allocated for.  Setting u~ invalidates the decoded u^ chain from that
 * level up, which the next residual or decode rebuilds.  Errors: CMG_EINVAL for
 * a bad context, which, level, width or NULL pointer; CMG_ECUDA; a pending
 * data-dependent error of earlier work (as cmg_sync). */
int64_t cmg_section_blocks(int dim, int level);
int cmg_section_width(const cmg_ctx *ctx, int which, int level);
cmg_status cmg_get_section(cmg_ctx *ctx, int which, int level, uint32_t *words_host,
                           int8_t *exps_host);
cmg_status cmg_set_section(cmg_ctx *ctx, int which, int level, int W,
                           const uint32_t *words_host, const int8_t *exps_host);

/* Decode the standard representation u^_L (eq. compact-to-standard) of planes
 * z0 .. z0+nz-1 of the current finest level into out_dev (nz * n * n doubles,
 * dense, device memory of the caller; n = 2^L - 1; in 2-D z0 = 0, nz = 1).
 * Values needing more than 53 bits are rounded to nearest by the conversion.
 * Synchronises.  Errors: CMG_EINVAL before cmg_start, for a NULL out_dev or
 * for planes outside 0..n-1; CMG_ECORRUPT / CMG_ERANGE for an invalid code or
 * an out-of-range value in the sections. */
cmg_status cmg_decode_solution(cmg_ctx *ctx, int64_t z0, int64_t nz, double *out_dev);

/* Checkpoint of the compact solution state (level, widths, sections of u~),
 * in host memory of the caller; both calls synchronise.  cmg_state_save with
 * buf == NULL returns the needed size in *len, and CMG_EINVAL when *len is
 * smaller than that.  cmg_state_load accepts only a checkpoint written by a
 * context with identical cmg_params (CMG_EINVAL otherwise, or when the buffer
 * is truncated) and resumes the FMG at the saved level, with the corrections
 * y~ zero; it may be called on a fresh context.  cmg_state_save returns
 * CMG_EINVAL before cmg_start. */
cmg_status cmg_state_save(cmg_ctx *ctx, void *buf, size_t *len);
cmg_status cmg_state_load(cmg_ctx *ctx, const void *buf, size_t len);

/* ---------------------------------------------------------------------------
 * Decoding without device allocation.  The paper has no counterpart to this
 * entry point; it serves callers that may not allocate device memory while
 * they run, e.g. an application that gives all of its device memory to its own
 * pool at start-up, or a time-critical loop that cannot accept the implicit
 * device-wide synchronisation of cudaMalloc/cudaFree.
 *
 * cmg_decode_compact computes the standard representation u^_L of planes
 * z0 .. z0+nz-1 (eq. compact-to-standard) from the sections u~_1 .. u~_L of a
 * compact vector, exactly like cmg_decode_solution, but without a context:
 * words_dev[l-1], exps_dev[l-1] and widths[l-1] describe section l in the BFP
 * layout above (device memory of the caller; the pointer arrays and widths are
 * host arrays), out_dev receives nz * n * n doubles (n = 2^L - 1; 2-D: z0 = 0,
 * nz = 1).  The decoded coarse levels it needs are kept in one static device
 * array of CMG_STATIC_SCRATCH_BYTES that every GPU loading this library holds
 * until the process exits; the call itself allocates nothing.
 *  - Capacity: returns CMG_ERANGE without launching anything when
 *    cmg_decode_compact_scratch_bytes(dim, L) exceeds CMG_STATIC_SCRATCH_BYTES
 *    (3-D up to L = 8, 2-D up to L = 11).
 *  - Every call looks up the array's device address with the caller's device
 *    current (a host-side query, not cached, so that a device reset cannot
 *    leave a stale address behind).  The first call on a device also makes the
 *    runtime load the array; make that first call before any stream capture.
 *  - All calls on one device share the array, which keeps the previous call's
 *    contents (the call clears what must start at zero).  Calls whose work may
 *    overlap on the GPU (different streams, or different host threads) race on
 *    the array and must be serialised by the caller.
 *  - Synchronises the stream; CMG_ECORRUPT / CMG_ERANGE / CMG_EINVAL as for
 *    cmg_decode_solution. */
#define CMG_STATIC_SCRATCH_BYTES ((size_t)24 << 20)
size_t cmg_decode_compact_scratch_bytes(int dim, int L);
cmg_status cmg_decode_compact(int dim, int L, const uint32_t *const *words_dev,
                              const int8_t *const *exps_dev, const int *widths, int64_t z0,
                              int64_t nz, double *out_dev, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Analytic storage model (Secs. 6.1.1 and 6.1.4 of the paper: mantissas of regressive-
 * precision vectors, and the comparison with progressive-precision FMG in BFP
 * arithmetic, "BFPMG").  Host-only arithmetic; no device work.
 *
 * Levels are this library's: level l = 1..L has n_l = (2^l - 1)^dim interior
 * DoF (the paper's level l - 1).  A regressive(+k, b) vector has k (L - l) + b
 * bits per value on level l (eq. regressive), a progressive(+k, b) one
 * k (l - 1) + b.  Mantissa bits only (sign included); exponents, padding and
 * the sublinear temporaries are not counted (the paper calls them negligible or
 * sublinear).  With k_u = p + 1 and k_r = m:
 *   cmg_vector  = sum_l n_l (k_u (L - l) + b1)                     (u~)
 *   cmg_fmg     = cmg_vector + 2 sum_l n_l (k_r (L - l) + b2)      (u~, r, y~)
 *   bfpmg_vector = n_L (k_u (L - 1) + b1)                          (u_L)
 *   bfpmg_fmg   = bfpmg_vector + n_L (k_r (L - 1) + b2)            (r_L)
 *               + n_(L-1) (k_r (L - 2) + b2)                       (r_(L-1))
 *               + sum_l n_l (k_r (l - 1) + b2)                     (y_1..L)
 * following the paper's assumptions for BFPMG (memory only for u_L, r_L,
 * r_(L-1) and y; matrices and right-hand side on the fly; same increments and
 * constants as CMG).  Savings are the BFPMG / CMG ratios.
 * Returns CMG_EINVAL for dim outside 1..3, L outside 1..40 or negative /
 * zero widths. */
typedef struct {
  double dofs;               /* n_L */
  double cmg_vector_bits, cmg_fmg_bits;
  double bfpmg_vector_bits, bfpmg_fmg_bits;
  double vector_saving, fmg_saving;
} cmg_storage;
cmg_status cmg_storage_model(int dim, int L, int k_u, int k_r, int b1, int b2, cmg_storage *out);

#ifdef __cplusplus
}
#endif
#endif /* CMG_H */
