// Host driver and C ABI of the compact FMG library (see include/cmg.h).
//
// The driver owns the compact hierarchy on the device and enqueues the kernels
// of cmg_kernels.cu on one CUDA stream.  Nothing here computes method
// arithmetic on the host except the load value at the single level-1 node and
// the Jacobi constants; every sweep over a grid runs in a kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cmg.h"
#include "cmg_device.cuh"
#include "cmg_kernels.h"

using namespace cmg;

namespace {

constexpr int MAXL = 14;
constexpr int META_CAP = 1 << 20;  // ints in the metadata pool (2 per section write)

struct SecBuf {
  uint32_t *words = nullptr;
  int8_t *exps = nullptr;
  size_t cap_words = 0;  // allocated words
  int W = 0;
  int *meta = nullptr;   // current metadata slot
};

struct Level {
  Geo g{};
  SecBuf u, u_alt, r, rc, y[2];
  int ycur = 0;
  bool y_zero = true;
  SecBuf t;                       // t^_l of the restriction chain (no pre-smoothing)
  long long *uh = nullptr, *w = nullptr, *acc = nullptr;
  int *uhg = nullptr, *wg = nullptr;  // per-block descriptors of u^_l and w_l
  int *accmeta = nullptr;
};

struct KStat {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  bool borrowed = false;  // ev holds the events of the solve's CUDA graph (not ours to destroy)
  double bytes = 0;
  double ms = 0;
  long long launches = 0;
};

// The whole FMG solve as one CUDA graph.  The host logic of a solve depends only
// on the context's inputs and configuration, never on device data, so a solve
// captured once replays with the same kernels and arguments; the host state at
// the end of the captured solve (buffer roles, widths, metadata slots, counters)
// is put back before each launch of the graph.
struct SolveGraph {
  cudaGraphExec_t exec = nullptr;
  bool capturing = false;
  bool failed = false;  // a capture of the current inputs failed: solve eagerly
  int warm = 0;         // eager solves of the current inputs
  long long captures = 0, graph_solves = 0;
  Level lv[MAXL + 1];
  int L = 0, uh_upto = 0, meta_next = 1, fb_next = 0;
  long long fast_ctas = 0, fast_ctas_top = 0, launches = 0;
  double alg_bytes = 0;
  std::vector<char> fb_top;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[CMG_KIND_COUNT][2];  // recorded by the graph
  long long k_launches[CMG_KIND_COUNT][2] = {};
  double k_bytes[CMG_KIND_COUNT][2] = {};
};

}  // namespace

struct cmg_ctx {
  cmg_params P{};
  cudaStream_t st = nullptr;
  int L = 0;
  Level lv[MAXL + 1];
  int *meta_pool = nullptr;
  int meta_next = 1;  // slot 0 stays all-zero: the metadata of an all-zero section
  int *err = nullptr;
  int32_t *tables = nullptr;
  size_t tables_cap = 0;  // int32 entries allocated for the tables
  int nterms = 0, scale_exp = 0, fsh = 0, rhs_bits = 0;
  std::vector<int32_t> tables_host;
  bool have_rhs = false;
  int uh_upto = 0;  // u^_1 .. u^_uh_upto agree with the current u~
  // exact Poisson path: on the finest FMG level (L = L_max) the level-(L-1)
  // sources w and u^ are read in two levels (section + P of level L-2), so that
  // level L_max - 1 holds no int64 copy of them
  bool tl = false, tl_capable = false;
  int c_num2 = 0, c_exp2 = 0;  // omega / (2d) = c_num2 2^c_exp2 (level-free part)
  std::string msg;
  int timing = 0;  // per-launch CUDA events: 0 none, 1 every launch, 2 launches on level L_max only
  const float *kfield = nullptr;  // diffusion: borrowed nodal coefficient
  const double *grhs = nullptr;   // diffusion: borrowed nodal right-hand side, or null
  int grhs_log2 = 0;              // its power-of-two scale: f_L = h_L^d 2^grhs_log2 g
  void *dbuf = nullptr;           // diffusion: d = rc - A y~ of the finest level in the cycle's type
  KStat stats[CMG_KIND_COUNT][2];  // per kernel kind; [1] = launches on level L_max
  long long launches = 0;
  double alg_bytes = 0;
  // specialised 3-D kernels (cmg_fast.cu): on by default for the exact path
  bool fast = true;
  unsigned *fb_tiles = nullptr;  // fallback tile list (one level's worth of tiles)
  int *fb_counts = nullptr;      // one zeroed count per specialised launch, FB_SLOTS in all
  int fb_next = 0;
  long long fast_ctas = 0, fast_ctas_top = 0;   // CTAs of specialised launches since cmg_start
  long long fb_done = 0, fb_done_top = 0;       // fallback tiles of slots already summed
  std::vector<char> fb_top;                     // slot on level L_max?
  bool graphs = true;  // solve through a CUDA graph where the stream allows (cmg_set_graphs)
  SolveGraph gr;
};

constexpr int FB_SLOTS = 4096;

// whether a new exact Poisson context starts on the two-level path
// (cmg_set_two_level): off, since the materialized sources are faster (the
// kernels are bound by instruction issue, not by the bytes the two-level path
// saves)
#ifndef CMG_TWO_LEVEL_DEFAULT
#define CMG_TWO_LEVEL_DEFAULT 0
#endif

// ---------------------------------------------------------------- helpers
static cmg_status fail(cmg_ctx *c, cmg_status s, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->msg = buf;
  }
  return s;
}

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(ctx, CMG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static Geo make_geo(int dim, int l) {
  Geo g;
  g.l = l;
  g.n = (1 << l) - 1;
  g.nz = dim == 3 ? g.n : 1;
  g.nbx = (g.n + 31) / 32;
  g.R = 32 * g.nbx;
  g.nblocks = (long long)g.nz * g.n * g.nbx;
  return g;
}

static int Wu(const cmg_ctx *c, int l, int L) { return c->P.k_u * (L - l) + c->P.b1; }
static int Wr(const cmg_ctx *c, int l, int L) { return c->P.k_r * (L - l) + c->P.b2; }

static int *new_meta(cmg_ctx *c) {
  if (c->meta_next >= META_CAP / 2) return nullptr;
  return c->meta_pool + 2 * (c->meta_next++);
}

static int bitlen_int(int v) {
  int b = 0;
  while (v) {
    b++;
    v >>= 1;
  }
  return b;
}

// Jacobi factor on level l: c_l = omega / (2d h_l^(d-2)) = c_num 2^c_exp
static void jacobi_factor(const cmg_ctx *c, int l, int &num, int &ex, int &bits) {
  num = c->c_num2;
  ex = c->c_exp2 + (c->P.dim - 2) * l;
  bits = bitlen_int(num);
}

static Sec sec_of(const SecBuf &b) {
  Sec s;
  s.words = b.words;
  s.exps = b.exps;
  s.W = b.W;
  s.meta = b.meta;
  return s;
}

static Tmp tmp_of(long long *v, int *gb, int *meta) {
  Tmp t;
  t.v = v;
  t.gb = gb;
  t.meta = meta;
  return t;
}

static cmg_status launched(cmg_ctx *ctx, double bytes) {
  ctx->launches++;
  ctx->alg_bytes += bytes;
  CU(cudaGetLastError());
  return CMG_OK;
}

static double sec_bytes(const Geo &g, int W) { return (double)g.nblocks * (4.0 * W + 1.0); }
static double tmp_bytes(const Geo &g) { return 8.0 * (double)g.nz * g.n * g.n; }

// inside a capture the record becomes an event-record node of the graph
static void ev_record(cmg_ctx *c, cudaEvent_t e) {
  if (c->gr.capturing) cudaEventRecordWithFlags(e, c->st, cudaEventRecordExternal);
  else cudaEventRecord(e, c->st);
}

// whether launches counted in k get events (stats[kind][1] holds the level-L_max launches)
static bool ev_on(const cmg_ctx *c, const KStat &k) {
  return c->timing == 1 || (c->timing == 2 && ((&k - &c->stats[0][0]) & 1) != 0);
}

static void ev_begin(cmg_ctx *c, KStat &k) {
  if (!ev_on(c, k)) return;
  if (k.ev.size() > 100000) return;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  ev_record(c, a);
  k.ev.push_back({a, b});
}

static void ev_end(cmg_ctx *c, KStat &k, double bytes) {
  k.launches++;
  k.bytes += bytes;
  if (!ev_on(c, k) || k.ev.empty() || k.ev.size() > 100000) return;
  ev_record(c, k.ev.back().second);
}

// statistics slot of a kernel launch on level l
static KStat &kstat(cmg_ctx *c, int kind, int l) { return c->stats[kind][l == c->P.L_max ? 1 : 0]; }

static void ev_collect(KStat &k) {
  for (auto &p : k.ev) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) k.ms += ms;
    if (!k.borrowed) {
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
  }
  k.ev.clear();
  k.borrowed = false;
}

static void stat_reset(KStat &k) {
  ev_collect(k);
  k.ms = 0;
  k.bytes = 0;
  k.launches = 0;
}

// ---------------------------------------------------------------- solve graph
// Drops the captured graph (its events too) and the count of eager solves.  Every
// launch of the graph has completed: cmg_fmg_solve synchronises before it returns.
static void graph_drop(cmg_ctx *c) {
  SolveGraph &g = c->gr;
  for (int k = 0; k < CMG_KIND_COUNT; k++)
    for (int t = 0; t < 2; t++) {
      if (c->stats[k][t].borrowed) ev_collect(c->stats[k][t]);  // the last launch's times stay
      for (auto &p : g.ev[k][t]) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
      }
      g.ev[k][t].clear();
    }
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  g.warm = 0;
  g.failed = false;
}

// an input or the configuration of the solve changed: the graph no longer applies
static void graph_touch(cmg_ctx *c) {
  if (c->gr.exec || c->gr.warm || c->gr.failed) graph_drop(c);
}

// the legacy default stream cannot be captured
static bool graph_usable(const cmg_ctx *c) {
  return c->graphs && c->st != nullptr && c->st != cudaStreamLegacy && !c->gr.failed;
}

// the host state at the end of the captured solve, and its statistics
static void graph_save(cmg_ctx *c) {
  SolveGraph &g = c->gr;
  for (int l = 0; l <= MAXL; l++) g.lv[l] = c->lv[l];
  g.L = c->L;
  g.uh_upto = c->uh_upto;
  g.meta_next = c->meta_next;
  g.fb_next = c->fb_next;
  g.fb_top = c->fb_top;
  g.fast_ctas = c->fast_ctas;
  g.fast_ctas_top = c->fast_ctas_top;
  g.launches = c->launches;
  g.alg_bytes = c->alg_bytes;
  for (int k = 0; k < CMG_KIND_COUNT; k++)
    for (int t = 0; t < 2; t++) {
      KStat &s = c->stats[k][t];
      g.ev[k][t] = std::move(s.ev);
      s.ev = g.ev[k][t];
      s.borrowed = true;
      g.k_launches[k][t] = s.launches;
      g.k_bytes[k][t] = s.bytes;
    }
}

static void graph_restore(cmg_ctx *c) {
  const SolveGraph &g = c->gr;
  for (int l = 0; l <= MAXL; l++) c->lv[l] = g.lv[l];
  c->L = g.L;
  c->uh_upto = g.uh_upto;
  c->meta_next = g.meta_next;
  c->fb_next = g.fb_next;
  c->fb_top = g.fb_top;
  c->fast_ctas = g.fast_ctas;
  c->fast_ctas_top = g.fast_ctas_top;
  c->fb_done = c->fb_done_top = 0;
  c->launches = g.launches;
  c->alg_bytes = g.alg_bytes;
  for (int k = 0; k < CMG_KIND_COUNT; k++)
    for (int t = 0; t < 2; t++) {
      KStat &s = c->stats[k][t];
      s.ev = g.ev[k][t];
      s.borrowed = true;
      s.launches = g.k_launches[k][t];
      s.bytes = g.k_bytes[k][t];
    }
}

// ---------------------------------------------------------------- validation
extern "C" cmg_status cmg_params_check(const cmg_params *p) {
  if (!p) return CMG_EINVAL;
  if (p->dim != 2 && p->dim != 3) return CMG_EINVAL;
  if (p->L_max < 1 || p->L_max > MAXL) return CMG_EINVAL;
  {  // block and plane indices of the finest level are 32-bit in the kernels
    const long long n = (1ll << p->L_max) - 1, nbx = (n + 31) / 32;
    if ((p->dim == 3 ? n : 1) * n * nbx >= (1ll << 31)) return CMG_ERANGE;
  }
  if (p->b1 < 2 || p->b2 < 2 || p->k_u < 0 || p->k_r < 0) return CMG_EINVAL;
  if (p->k_u * (p->L_max - 1) + p->b1 > 32 || p->k_r * (p->L_max - 1) + p->b2 > 32) return CMG_ERANGE;
  if (p->N_ir < 1 || p->nu1 < 0 || p->nu2 < 1 || p->nu1 > 64 || p->nu2 > 64) return CMG_EINVAL;
  // without pre-smoothing the restriction chain carries t^ at (p+1)L + b1 bits
  if (p->nu1 == 0 && p->k_u * p->L_max + p->b1 > 32) return CMG_ERANGE;
  if (p->omega_num <= 0 || p->omega_log2den < 0 || p->omega_log2den > 30) return CMG_EINVAL;
  if (p->arith != CMG_ARITH_EXACT && p->arith != CMG_ARITH_FP32 && p->arith != CMG_ARITH_FP64) return CMG_EINVAL;
  if (p->coef != CMG_COEF_POISSON && p->coef != CMG_COEF_DIFFUSION) return CMG_EINVAL;
  if (p->coef == CMG_COEF_DIFFUSION && (p->arith == CMG_ARITH_EXACT || p->nu1 < 1)) return CMG_EINVAL;
  if (p->smoother != CMG_SMOOTHER_JACOBI &&
      (p->smoother != CMG_SMOOTHER_RBGS || p->nu1 != 0 || p->coef != CMG_COEF_POISSON))
    return CMG_EINVAL;
  if (p->dim == 3 && p->omega_num % 3 != 0) return CMG_EINVAL;  // omega/6 must be dyadic
  // keep the Jacobi numerator small (it widens the exact integers by its bit length)
  int num = p->dim == 3 ? p->omega_num / 3 : p->omega_num;
  while (num % 2 == 0) num /= 2;
  if (num >= (1 << 10)) return CMG_EINVAL;
  if (p->arith == CMG_ARITH_FP32) {
    // binary32 must hold every r~ / y~ code exactly, and c rc of the fused first sweep
    int cb = 0;
    for (int t = num; t; t >>= 1) cb++;
    if (p->k_r * (p->L_max - 1) + p->b2 + cb > 24) return CMG_ERANGE;
  }
  return CMG_OK;
}

// ---------------------------------------------------------------- lifetime
static cmg_status alloc_sec(cmg_ctx *ctx, SecBuf &b, const Geo &g, int Wmax) {
  b.cap_words = (size_t)g.nblocks * Wmax;
  CU(cudaMalloc(&b.words, b.cap_words * sizeof(uint32_t)));
  // whole 16-byte units: the two-level staging copies the aligned word around an exponent
  CU(cudaMalloc(&b.exps, ((size_t)g.nblocks + 15) & ~(size_t)15));
  b.W = Wmax;
  b.meta = ctx->meta_pool;  // slot 0: empty
  return CMG_OK;
}

static void free_sec(SecBuf &b) {
  cudaFree(b.words);
  cudaFree(b.exps);
  b.words = nullptr;
  b.exps = nullptr;
}

extern "C" void cmg_destroy(cmg_ctx *ctx) {
  if (!ctx) return;
  graph_drop(ctx);
  for (int l = 1; l <= MAXL; l++) {
    Level &v = ctx->lv[l];
    free_sec(v.u);
    free_sec(v.u_alt);
    free_sec(v.r);
    free_sec(v.rc);
    free_sec(v.y[0]);
    free_sec(v.y[1]);
    free_sec(v.t);
    cudaFree(v.uh);
    cudaFree(v.w);
    cudaFree(v.acc);
    cudaFree(v.uhg);
    cudaFree(v.wg);
  }
  for (int k = 0; k < CMG_KIND_COUNT; k++) {
    stat_reset(ctx->stats[k][0]);
    stat_reset(ctx->stats[k][1]);
  }
  cudaFree(ctx->dbuf);
  cudaFree(ctx->fb_tiles);
  cudaFree(ctx->fb_counts);
  cudaFree(ctx->meta_pool);
  cudaFree(ctx->err);
  cudaFree(ctx->tables);
  delete ctx;
}

extern "C" cmg_status cmg_create(const cmg_params *p, void *stream, cmg_ctx **out) {
  if (!out) return CMG_EINVAL;
  *out = nullptr;
  cmg_status s = cmg_params_check(p);
  if (s != CMG_OK) return s;
  cmg_ctx *ctx = new (std::nothrow) cmg_ctx();
  if (!ctx) return CMG_ENOMEM;
  ctx->P = *p;
  ctx->st = (cudaStream_t)stream;
  ctx->tl_capable = p->arith == CMG_ARITH_EXACT && p->coef == CMG_COEF_POISSON && p->L_max >= 3;
  ctx->tl = ctx->tl_capable && CMG_TWO_LEVEL_DEFAULT;
  {
    int num = p->dim == 3 ? p->omega_num / 3 : p->omega_num;
    int ex = -p->omega_log2den - (p->dim == 3 ? 1 : 2);  // 2-D: /4; 3-D: /6 = /3 /2
    while (num % 2 == 0) {
      num /= 2;
      ex++;
    }
    ctx->c_num2 = num;
    ctx->c_exp2 = ex;
  }
  cmg_status r = CMG_OK;
  auto chk = [&](cudaError_t e) {
    if (e != cudaSuccess && r == CMG_OK) r = fail(ctx, e == cudaErrorMemoryAllocation ? CMG_ENOMEM : CMG_ECUDA,
                                                  "allocation: %s", cudaGetErrorString(e));
  };
  chk(cudaMalloc(&ctx->meta_pool, META_CAP * sizeof(int)));
  chk(cudaMalloc(&ctx->err, 8 * sizeof(int)));
  if (r == CMG_OK) {
    chk(cudaMemsetAsync(ctx->meta_pool, 0, META_CAP * sizeof(int), ctx->st));
    chk(cudaMemsetAsync(ctx->err, 0, 8 * sizeof(int), ctx->st));
  }
  if (r == CMG_OK && p->dim == 3 && p->arith == CMG_ARITH_EXACT) {
    // fallback tiles of the specialised kernels: at most every tile of the finest level
    const Geo g = make_geo(3, p->L_max);
    const size_t tiles = (size_t)g.nbx * ((g.n + TY - 1) / TY) * ((g.nz + ZC - 1) / ZC);
    chk(cudaMalloc(&ctx->fb_tiles, tiles * sizeof(unsigned)));
    chk(cudaMalloc(&ctx->fb_counts, FB_SLOTS * sizeof(int)));
    if (r == CMG_OK) chk(cudaMemsetAsync(ctx->fb_counts, 0, FB_SLOTS * sizeof(int), ctx->st));
  }
  for (int l = 1; l <= p->L_max && r == CMG_OK; l++) {
    Level &v = ctx->lv[l];
    v.g = make_geo(p->dim, l);
    const Geo &g = v.g;
    int wu = Wu(ctx, l, p->L_max), wr = Wr(ctx, l, p->L_max);
    if ((r = alloc_sec(ctx, v.u, g, wu)) != CMG_OK) break;
    if (l < p->L_max && (r = alloc_sec(ctx, v.u_alt, g, wu)) != CMG_OK) break;
    if ((r = alloc_sec(ctx, v.r, g, wr)) != CMG_OK) break;
    if (l < p->L_max && (r = alloc_sec(ctx, v.rc, g, wr)) != CMG_OK) break;
    if ((r = alloc_sec(ctx, v.y[0], g, wr)) != CMG_OK) break;
    if ((r = alloc_sec(ctx, v.y[1], g, wr)) != CMG_OK) break;
    // t^_l of the restriction chain (no pre-smoothing): the finest level restricts
    // its t^ inside the residual kernel and needs none
    if (p->nu1 == 0 && l < p->L_max && (r = alloc_sec(ctx, v.t, g, p->k_u * p->L_max + p->b1)) != CMG_OK) break;
    if (l < p->L_max || l == 1) {
      size_t nt = (size_t)g.nz * g.n * g.R;
      // level L_max - 1 of the two-level path keeps its restriction accumulator only
      const bool temps = !(ctx->tl && l == p->L_max - 1);
      if (temps) {
        chk(cudaMalloc(&v.uh, nt * 8));
        chk(cudaMalloc(&v.w, nt * 8));
        chk(cudaMalloc(&v.uhg, (size_t)g.nblocks * sizeof(int)));
        chk(cudaMalloc(&v.wg, (size_t)g.nblocks * sizeof(int)));
      }
      chk(cudaMalloc(&v.acc, nt * 8));
      if (r == CMG_OK) {
        chk(cudaMemsetAsync(v.acc, 0, nt * 8, ctx->st));
        if (temps) {
          chk(cudaMemsetAsync(v.uh, 0, nt * 8, ctx->st));
          chk(cudaMemsetAsync(v.w, 0, nt * 8, ctx->st));
        }
      }
    }
  }
  if (r != CMG_OK) {
    cmg_destroy(ctx);
    return r;
  }
  *out = ctx;
  return CMG_OK;
}

extern "C" const char *cmg_last_error(const cmg_ctx *ctx) { return ctx ? ctx->msg.c_str() : "null context"; }

extern "C" cmg_status cmg_set_timing(cmg_ctx *ctx, int mode) {
  if (!ctx || mode < 0 || mode > 2) return CMG_EINVAL;
  if (ctx->timing != mode) graph_touch(ctx);
  ctx->timing = mode;
  return CMG_OK;
}

extern "C" cmg_status cmg_set_fast_kernels(cmg_ctx *ctx, int enable) {
  if (!ctx) return CMG_EINVAL;
  if (ctx->fast != (enable != 0)) graph_touch(ctx);
  ctx->fast = enable != 0;
  return CMG_OK;
}

extern "C" cmg_status cmg_set_graphs(cmg_ctx *ctx, int enable) {
  if (!ctx) return CMG_EINVAL;
  if (!enable) graph_drop(ctx);
  ctx->graphs = enable != 0;
  return CMG_OK;
}

extern "C" cmg_status cmg_graph_stats(const cmg_ctx *ctx, int64_t *captures, int64_t *graph_solves) {
  if (!ctx) return CMG_EINVAL;
  if (captures) *captures = ctx->gr.captures;
  if (graph_solves) *graph_solves = ctx->gr.graph_solves;
  return CMG_OK;
}

// the int64 u^ and w of level L_max - 1 (and their block descriptors)
static void free_top_temps(cmg_ctx *ctx) {
  Level &v = ctx->lv[ctx->P.L_max - 1];
  cudaFree(v.uh);
  cudaFree(v.w);
  cudaFree(v.uhg);
  cudaFree(v.wg);
  v.uh = v.w = nullptr;
  v.uhg = v.wg = nullptr;
}

static cmg_status alloc_top_temps(cmg_ctx *ctx) {
  Level &v = ctx->lv[ctx->P.L_max - 1];
  const Geo &g = v.g;
  const size_t nt = (size_t)g.nz * g.n * g.R;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&v.uh, nt * 8);
  if (e == cudaSuccess) e = cudaMalloc(&v.w, nt * 8);
  if (e == cudaSuccess) e = cudaMalloc(&v.uhg, (size_t)g.nblocks * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&v.wg, (size_t)g.nblocks * sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(v.uh, 0, nt * 8, ctx->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.w, 0, nt * 8, ctx->st);
  if (e != cudaSuccess) {
    free_top_temps(ctx);
    return fail(ctx, e == cudaErrorMemoryAllocation ? CMG_ENOMEM : CMG_ECUDA, "allocation: %s",
                cudaGetErrorString(e));
  }
  return CMG_OK;
}

extern "C" cmg_status cmg_set_two_level(cmg_ctx *ctx, int enable) {
  if (!ctx) return CMG_EINVAL;
  const bool on = enable != 0;
  if (on && !ctx->tl_capable)
    return fail(ctx, CMG_EUNSUPPORTED, "two-level sources need the exact Poisson path and L_max >= 3");
  if (on == ctx->tl) return CMG_OK;
  CU(cudaStreamSynchronize(ctx->st));  // no launch in flight reads the buffers
  graph_touch(ctx);
  if (on) {
    free_top_temps(ctx);
  } else {
    cmg_status s = alloc_top_temps(ctx);
    if (s) return s;
  }
  ctx->tl = on;
  // u^ of level L_max - 1 is not materialized on the two-level path, and not yet
  // on the other one
  ctx->uh_upto = std::min(ctx->uh_upto, ctx->P.L_max - 2);
  return CMG_OK;
}

// sums the fallback counts of the slots used so far into fb_done (synchronises)
static cmg_status fb_collect(cmg_ctx *ctx) {
  if (!ctx->fb_counts || ctx->fb_next == 0) return CMG_OK;
  std::vector<int> c(ctx->fb_next);
  CU(cudaStreamSynchronize(ctx->st));
  CU(cudaMemcpy(c.data(), ctx->fb_counts, c.size() * sizeof(int), cudaMemcpyDeviceToHost));
  for (int k = 0; k < ctx->fb_next; k++) {
    ctx->fb_done += c[k];
    if (ctx->fb_top[k]) ctx->fb_done_top += c[k];
  }
  CU(cudaMemsetAsync(ctx->fb_counts, 0, FB_SLOTS * sizeof(int), ctx->st));
  ctx->fb_next = 0;
  return CMG_OK;
}

// a zeroed fallback count for the next specialised launch on level l (the slots
// are summed and cleared together, once every FB_SLOTS launches)
static cmg_status fb_slot(cmg_ctx *ctx, int l, int **slot) {
  if (ctx->fb_next >= FB_SLOTS) {
    cmg_status s = fb_collect(ctx);
    if (s) return s;
  }
  if ((int)ctx->fb_top.size() < FB_SLOTS) ctx->fb_top.resize(FB_SLOTS);
  ctx->fb_top[ctx->fb_next] = l == ctx->P.L_max;
  *slot = ctx->fb_counts + ctx->fb_next++;
  return CMG_OK;
}

static long long tiles_of(const Geo &g) {
  return (long long)g.nbx * ((g.n + TY - 1) / TY) * ((g.nz + ZC - 1) / ZC);
}

extern "C" cmg_status cmg_fast_stats(cmg_ctx *ctx, int top, int64_t *ctas, int64_t *fallback_ctas) {
  if (!ctx || top < 0 || top > 1) return CMG_EINVAL;
  cmg_status s = fb_collect(ctx);
  if (s) return s;
  if (ctas) *ctas = top ? ctx->fast_ctas_top : ctx->fast_ctas;
  if (fallback_ctas) *fallback_ctas = top ? ctx->fb_done_top : ctx->fb_done;
  return CMG_OK;
}

extern "C" int cmg_level(const cmg_ctx *ctx) { return ctx ? ctx->L : -1; }

extern "C" int64_t cmg_section_blocks(int dim, int level) {
  if ((dim != 2 && dim != 3) || level < 1 || level > MAXL) return -1;
  return make_geo(dim, level).nblocks;
}

// ---------------------------------------------------------------- coefficient
extern "C" cmg_status cmg_set_coefficient(cmg_ctx *ctx, const float *k_dev, int64_t n) {
  if (!ctx || !k_dev) return CMG_EINVAL;
  if (ctx->P.coef != CMG_COEF_DIFFUSION) return fail(ctx, CMG_EINVAL, "coefficient on a Poisson context");
  const long long N = (1ll << ctx->P.L_max) + 1;
  if (n != (ctx->P.dim == 3 ? N * N * N : N * N)) return fail(ctx, CMG_EINVAL, "coefficient size");
  if (k_dev != ctx->kfield) graph_touch(ctx);  // the graph reads the field through its pointer
  ctx->kfield = k_dev;
  if (!ctx->dbuf) {
    const Geo g = make_geo(ctx->P.dim, ctx->P.L_max);
    const size_t es = ctx->P.arith == CMG_ARITH_FP64 ? sizeof(double) : sizeof(float);
    CU(cudaMalloc(&ctx->dbuf, (size_t)g.nz * g.n * g.R * es));
  }
  return CMG_OK;
}

extern "C" cmg_status cmg_set_rhs_nodal(cmg_ctx *ctx, const double *g_dev, int64_t n, int scale_log2) {
  if (!ctx || !g_dev) return CMG_EINVAL;
  if (ctx->P.coef != CMG_COEF_DIFFUSION) return fail(ctx, CMG_EINVAL, "nodal right-hand side on a Poisson context");
  const long long n1 = (1ll << ctx->P.L_max) - 1;
  if (n != (ctx->P.dim == 3 ? n1 * n1 * n1 : n1 * n1)) return fail(ctx, CMG_EINVAL, "right-hand side size");
  if (scale_log2 < -512 || scale_log2 > 512) return fail(ctx, CMG_EINVAL, "right-hand side scale 2^%d", scale_log2);
  if (g_dev != ctx->grhs || scale_log2 != ctx->grhs_log2 || !ctx->have_rhs) graph_touch(ctx);
  ctx->grhs = g_dev;
  ctx->grhs_log2 = scale_log2;
  ctx->have_rhs = true;
  return CMG_OK;
}

extern "C" cmg_status cmg_gradient(cmg_ctx *ctx, const double *u_dev, const double *lam_dev, double *dk_dev,
                                   double *dg_dev) {
  if (!ctx || !u_dev || !lam_dev || !dk_dev) return CMG_EINVAL;
  if (ctx->P.coef != CMG_COEF_DIFFUSION) return fail(ctx, CMG_EINVAL, "gradient needs the diffusion problem");
  GradArgs a{};
  a.dim = ctx->P.dim;
  a.L = ctx->P.L_max;
  a.u = u_dev;
  a.lam = lam_dev;
  a.kfield = ctx->kfield;
  a.kN = (1 << ctx->P.L_max) + 1;
  a.dk = dk_dev;
  a.dg = dg_dev;
  launch_gradient(a, ctx->st);
  CU(cudaGetLastError());
  return CMG_OK;
}

// ---------------------------------------------------------------- right-hand side
extern "C" cmg_status cmg_set_rhs_separable(cmg_ctx *ctx, int nterms, const int32_t *tab, int scale_exp) {
  if (!ctx || !tab || nterms < 1 || nterms > 64) return CMG_EINVAL;
  const int d = ctx->P.dim, n1 = (1 << ctx->P.L_max) - 1;
  size_t cnt = (size_t)nterms * d * n1;
  unsigned __int128 bound = 0;
  for (int t = 0; t < nterms; t++) {
    unsigned __int128 prod = 1;
    for (int a = 0; a < d; a++) {
      long long m = 0;
      for (int i = 0; i < n1; i++) {
        long long v = std::llabs((long long)tab[((size_t)t * d + a) * n1 + i]);
        if (v > (1ll << 30)) return fail(ctx, CMG_EINVAL, "table entry above 2^30");
        m = std::max(m, v);
      }
      prod *= (unsigned __int128)m;
    }
    bound += prod;
  }
  int B = 0;
  for (unsigned __int128 t = bound; t; t >>= 1) B++;
  // the graph of the solve holds the table pointer and values derived from the
  // tables (the level-1 load): it stays only for the same tables
  const bool same = ctx->have_rhs && !ctx->grhs && nterms == ctx->nterms && scale_exp == ctx->scale_exp &&
                    ctx->tables_cap >= cnt && ctx->tables_host.size() == cnt &&
                    std::equal(tab, tab + cnt, ctx->tables_host.begin());
  if (!same) graph_touch(ctx);
  if (ctx->tables_cap < cnt) {  // the device buffer is kept across calls that fit in it
    cudaFree(ctx->tables);
    ctx->tables = nullptr;
    ctx->tables_cap = 0;
    CU(cudaMalloc(&ctx->tables, cnt * sizeof(int32_t)));
    ctx->tables_cap = cnt;
  }
  // the host copy is pageable, so the copy has taken the data when the call
  // returns and the caller's array is free at once (no stream synchronisation)
  ctx->tables_host.assign(tab, tab + cnt);
  CU(cudaMemcpyAsync(ctx->tables, ctx->tables_host.data(), cnt * sizeof(int32_t), cudaMemcpyHostToDevice,
                     ctx->st));
  ctx->nterms = nterms;
  ctx->scale_exp = scale_exp;
  ctx->fsh = B > 50 ? B - 50 : 0;
  ctx->rhs_bits = B;
  ctx->have_rhs = true;
  return CMG_OK;
}

// F_q at the level-1 node (coordinates 1/2): exact table product, RNE shift
static long long rhs_level1(const cmg_ctx *c) {
  const int d = c->P.dim, n1 = (1 << c->P.L_max) - 1, idx = (1 << (c->P.L_max - 1)) - 1;
  __int128 F = 0;
  for (int t = 0; t < c->nterms; t++) {
    __int128 p = 1;
    for (int a = 0; a < d; a++) p *= (__int128)c->tables_host[((size_t)t * d + a) * n1 + idx];
    F += p;
  }
  int s = c->fsh;
  if (s <= 0) return (long long)F;
  __int128 q = F >> s, rem = F - (q << s), half = (__int128)1 << (s - 1);
  if (rem > half || (rem == half && (q & 1))) q += 1;
  return (long long)q;
}

// ---------------------------------------------------------------- building blocks
static cmg_status set_zero_section(cmg_ctx *ctx, SecBuf &b, const Geo &g, int W) {
  b.W = W;
  b.meta = ctx->meta_pool;
  CU(cudaMemsetAsync(b.exps, 0x80, (size_t)g.nblocks, ctx->st));
  CU(cudaMemsetAsync(b.words, 0, (size_t)g.nblocks * W * sizeof(uint32_t), ctx->st));
  return CMG_OK;
}

static cmg_status fresh_tmp_meta(cmg_ctx *ctx, int *&slot) {
  slot = new_meta(ctx);
  if (!slot) return fail(ctx, CMG_ERANGE, "metadata pool exhausted");
  return CMG_OK;
}

static cmg_status fresh_meta(cmg_ctx *ctx, SecBuf &b) {
  b.meta = new_meta(ctx);
  if (!b.meta) return fail(ctx, CMG_ERANGE, "metadata pool exhausted");
  return CMG_OK;
}

static cmg_status run_chain(cmg_ctx *ctx, int upto) {
  if (ctx->tl && upto >= ctx->P.L_max - 1)  // that level has no u^ buffer on the two-level path
    return fail(ctx, CMG_EINVAL, "u^ of level %d is formed on the fly", upto);
  for (int l = 1; l <= upto; l++) {
    Level &v = ctx->lv[l];
    ChainArgs a{};
    a.g = v.g;
    a.gc = l > 1 ? ctx->lv[l - 1].g : v.g;
    a.u = sec_of(v.u);
    a.has_uhc = l > 1;
    if (l > 1) a.uhc = tmp_of(ctx->lv[l - 1].uh, ctx->lv[l - 1].uhg, nullptr);
    a.uh_out = tmp_of(v.uh, v.uhg, nullptr);
    a.err = ctx->err;
    ev_begin(ctx, kstat(ctx, CMG_KIND_OTHER, l));
    launch_chain(ctx->P.dim, a, ctx->st);
    ev_end(ctx, kstat(ctx, CMG_KIND_OTHER, l), sec_bytes(v.g, v.u.W) + tmp_bytes(v.g));
    cmg_status s = launched(ctx, sec_bytes(v.g, v.u.W) + tmp_bytes(v.g) + (l > 1 ? tmp_bytes(a.gc) : 0));
    if (s) return s;
  }
  return CMG_OK;
}

static Level &LV(cmg_ctx *c, int l) { return c->lv[l]; }

// the two-level sources are in use at the current FMG level
static bool tl_on(const cmg_ctx *c) { return c->tl && c->L == c->P.L_max; }

// w_(L-1) = y~_(L-1) + P w_(L-2) and u^_(L-1) = u~_(L-1) + P u^_(L-2) in two levels
static Tmp2 two_level(cmg_ctx *ctx, const SecBuf &s, bool w) {
  const Level &b = LV(ctx, ctx->L - 2);
  Tmp2 t{};
  t.s = sec_of(s);
  t.b = w ? tmp_of(b.w, b.wg, nullptr) : tmp_of(b.uh, b.uhg, nullptr);
  t.gb = b.g;
  return t;
}

// rc section of level l at the current FMG level
static SecBuf &rc_of(cmg_ctx *c, int l) {
  if (l == c->L) return c->lv[l].r;
  if (c->P.nu1 == 0) return c->lv[l].r;
  return c->lv[l].rc;
}

static cmg_status do_residual(cmg_ctx *ctx, bool first_sweep) {
  const int L = ctx->L, d = ctx->P.dim;
  const bool two = tl_on(ctx);  // u^_(L-1) = u~_(L-1) + P u^_(L-2) on the fly
  const int need = two ? L - 2 : L - 1;
  if (ctx->uh_upto < need) {
    cmg_status s = run_chain(ctx, need);
    if (s) return s;
    ctx->uh_upto = need;
  }
  Level &v = LV(ctx, L);
  ResidArgs a{};
  a.g = v.g;
  a.gc = L > 1 ? LV(ctx, L - 1).g : v.g;
  a.u = sec_of(v.u);
  a.has_uhc = L > 1;
  if (two) {
    a.tl = 1;
    a.uhc2 = two_level(ctx, LV(ctx, L - 1).u, false);
  } else if (L > 1) {
    a.uhc = tmp_of(LV(ctx, L - 1).uh, LV(ctx, L - 1).uhg, nullptr);
  }
  a.tables = ctx->tables;
  a.nterms = ctx->nterms;
  a.n1max = (1 << ctx->P.L_max) - 1;
  a.Lmax = ctx->P.L_max;
  a.fsh = ctx->fsh;
  a.rhs_bits = ctx->rhs_bits;
  a.Gf = ctx->scale_exp + ctx->fsh - d * L;
  v.r.W = Wr(ctx, L, L);
  cmg_status s = fresh_meta(ctx, v.r);
  if (s) return s;
  a.r_out = sec_of(v.r);
  const bool diff = ctx->P.coef == CMG_COEF_DIFFUSION;
  if (diff) {
    if (!ctx->kfield) return fail(ctx, CMG_EINVAL, "diffusion without a coefficient (cmg_set_coefficient)");
    first_sweep = false;  // the first sweep runs as a sweep with per-node factors
    a.kfield = ctx->kfield;
    a.kN = (1 << ctx->P.L_max) + 1;
    a.grhs = ctx->grhs;
    a.grhs_log2 = ctx->grhs_log2;
  }
  a.first_sweep = first_sweep;
  jacobi_factor(ctx, L, a.c_num, a.c_exp, a.cbits);
  if (first_sweep) {
    SecBuf &y = v.y[0];
    y.W = Wr(ctx, L, L);
    if ((s = fresh_meta(ctx, y))) return s;
    a.y_out = sec_of(y);
    v.ycur = 0;
    v.y_zero = false;
  }
  // without pre-smoothing, t^ (Table 1 width (p+1)L + b1) feeds the restriction
  // chain; on level L the kernel restricts it at once (R t^_L into acc_(L-1))
  const bool chain = ctx->P.nu1 == 0 && L > 1;
  const int Wt = ctx->P.k_u * L + ctx->P.b1;
  if (chain) {
    Level &c = LV(ctx, L - 1);
    a.fuse_restrict = 1;
    a.Wt = Wt;  // the rounding width of t^_L, which is not stored
    if ((s = fresh_tmp_meta(ctx, c.accmeta))) return s;
    a.racc = tmp_of(c.acc, nullptr, c.accmeta);
    for (int l = 1; l <= L; l++) {
      a.umeta[l] = LV(ctx, l).u.meta;
      a.uW[l] = LV(ctx, l).u.W;
    }
  }
  a.err = ctx->err;
  // the coarse source: u^_(L-1), or in two levels u~_(L-1) and u^_(L-2)
  const double src = two ? sec_bytes(a.gc, a.uhc2.s.W) + tmp_bytes(LV(ctx, L - 2).g) : (L > 1 ? tmp_bytes(a.gc) : 0);
  double bytes = sec_bytes(v.g, v.u.W) + src + sec_bytes(v.g, v.r.W) +
                 (first_sweep ? sec_bytes(v.g, v.r.W) : 0) + (chain ? 2 * tmp_bytes(a.gc) : 0);
  if (!diff && ctx->fast && ctx->fb_tiles) {
    a.tiles = ctx->fb_tiles;
    if ((s = fb_slot(ctx, L, &a.ntiles))) return s;
  }
  bool fast = false;
  ev_begin(ctx, kstat(ctx, CMG_KIND_RESIDUAL, L));
  if (diff) launch_residual_diffusion(d, a, ctx->st);
  else if (!(fast = a.tiles && launch_residual_fast(a, ctx->st))) launch_residual(d, a, ctx->st);
  ev_end(ctx, kstat(ctx, CMG_KIND_RESIDUAL, L), bytes);
  if (fast) {
    ctx->launches++;  // the generic kernel over the fallback tiles
    ctx->fast_ctas += tiles_of(v.g);
    if (L == ctx->P.L_max) ctx->fast_ctas_top += tiles_of(v.g);
  }
  if ((s = launched(ctx, bytes))) return s;
  if (chain) {  // t^_l = round(R t^_(l+1)), r_l = round(t^_l) (Algorithm 2)
    for (int l = L; l >= 2; l--) {
      Level &f = LV(ctx, l), &c = LV(ctx, l - 1);
      if (l < L) {  // level L was restricted by the residual kernel
        RestrictArgs ra{};
        ra.g = f.g;
        ra.gc = c.g;
        ra.has_y = 0;
        ra.rc = sec_of(f.t);
        if ((s = fresh_tmp_meta(ctx, c.accmeta))) return s;
        ra.acc = tmp_of(c.acc, nullptr, c.accmeta);
        ra.err = ctx->err;
        ev_begin(ctx, kstat(ctx, CMG_KIND_RESTRICT, l));
        launch_restrict(d, ra, ctx->st);
        ev_end(ctx, kstat(ctx, CMG_KIND_RESTRICT, l), sec_bytes(f.g, Wt) + 2 * tmp_bytes(c.g));
        if ((s = launched(ctx, sec_bytes(f.g, Wt) + 2 * tmp_bytes(c.g)))) return s;
      }
      AccArgs b{};
      b.g = c.g;
      b.acc = tmp_of(c.acc, nullptr, c.accmeta);
      c.r.W = Wr(ctx, l - 1, L);
      if ((s = fresh_meta(ctx, c.r))) return s;
      b.r_out = sec_of(c.r);
      b.chain = 1;
      c.t.W = Wt;
      if ((s = fresh_meta(ctx, c.t))) return s;
      b.t_out = sec_of(c.t);
      jacobi_factor(ctx, l - 1, b.c_num, b.c_exp, b.cbits);
      b.err = ctx->err;
      ev_begin(ctx, kstat(ctx, CMG_KIND_ACC_ENCODE, l));
      launch_acc_encode(d, b, ctx->st);
      ev_end(ctx, kstat(ctx, CMG_KIND_ACC_ENCODE, l), 2 * tmp_bytes(c.g) + sec_bytes(c.g, c.r.W) + sec_bytes(c.g, Wt));
      if ((s = launched(ctx, 2 * tmp_bytes(c.g) + sec_bytes(c.g, c.r.W) + sec_bytes(c.g, Wt)))) return s;
    }
  }
  return CMG_OK;
}

// one sweep (or, with rb, one colour's half-sweep) on level l reading y[ycur]
// (unless y_zero), writing y[1-ycur]
struct SweepOpts {
  bool has_z = false, write_y = true, corr = false, write_w = false, write_uh = false;
  int rb = 0;  // red-black half-sweep: 1 red nodes only, 2 black nodes only
};

static cmg_status do_sweep(cmg_ctx *ctx, int l, const SweepOpts &o_in) {
  const int L = ctx->L, d = ctx->P.dim;
  Level &v = LV(ctx, l);
  SweepOpts o = o_in;
  if (tl_on(ctx) && l == L - 1 && (o.write_w || o.write_uh)) {
    // level L-1 keeps y~' (the finest level reads w_(L-1) = y~' + P w_(L-2)) and no w, u^
    o.write_y = true;
    o.write_w = false;
    o.write_uh = false;
  }
  const bool two = tl_on(ctx) && l == L && o.has_z;  // z_L = P (y~_(L-1) + P w_(L-2))
  if (two && LV(ctx, L - 1).y_zero)
    return fail(ctx, CMG_EINVAL, "the finest up-sweep needs the level-%d up-sweep of the same cycle", L - 1);
  if ((o.write_w && !v.w) || (o.write_uh && !v.uh))  // level L_max - 1 of the two-level path
    return fail(ctx, CMG_EINVAL, "level %d keeps no int64 w or u^", l);
  SweepArgs a{};
  a.g = v.g;
  a.gc = l > 1 ? LV(ctx, l - 1).g : v.g;
  a.has_y = !v.y_zero;
  a.has_z = o.has_z;
  a.write_y = o.write_y;
  a.corr = o.corr;
  a.write_w = o.write_w;
  a.write_uh = o.write_uh;
  a.rb = o.rb;
  a.has_uhc = l > 1;
  a.Wy = Wr(ctx, l, L);
  if (a.has_y) a.y_in = sec_of(v.y[v.ycur]);
  a.rc = sec_of(rc_of(ctx, l));
  cmg_status s;
  SecBuf &yo = v.y[1 - v.ycur];
  if (o.write_y) {
    yo.W = a.Wy;
    if ((s = fresh_meta(ctx, yo))) return s;
    a.y_out = sec_of(yo);
  }
  if (o.corr) {
    a.u_in = sec_of(v.u);
    SecBuf un = v.u;  // in place: each block is read and rewritten by one warp
    un.W = Wu(ctx, l, L);
    if ((s = fresh_meta(ctx, un))) return s;
    a.u_out = sec_of(un);
    v.u.meta = un.meta;
    v.u.W = un.W;
  }
  if (two) {
    a.tl = 1;
    a.wc2 = two_level(ctx, LV(ctx, L - 1).y[LV(ctx, L - 1).ycur], true);
  } else if (o.has_z) {
    a.wc = tmp_of(LV(ctx, l - 1).w, LV(ctx, l - 1).wg, nullptr);
  }
  if (ctx->P.arith != CMG_ARITH_EXACT) {  // floating-point w temporaries in the same buffers
    if (o.has_z) a.wc_r = LV(ctx, l - 1).w;
    if (o.write_w) a.w_out_r = v.w;
  }
  if (ctx->P.coef == CMG_COEF_DIFFUSION) {
    a.kfield = ctx->kfield;
    a.kN = (1 << ctx->P.L_max) + 1;
    a.kstride = 1 << (ctx->P.L_max - l);
    a.omega = (float)ctx->P.omega_num / (float)(1 << ctx->P.omega_log2den);
  }
  if (l > 1 && !two) a.uhc = tmp_of(LV(ctx, l - 1).uh, LV(ctx, l - 1).uhg, nullptr);
  if (o.write_w) a.w_out = tmp_of(v.w, v.wg, nullptr);
  if (o.write_uh) a.uh_out = tmp_of(v.uh, v.uhg, nullptr);
  jacobi_factor(ctx, l, a.c_num, a.c_exp, a.cbits);
  a.err = ctx->err;
  // the coarse source: w_(l-1), or in two levels y~_(L-1) and w_(L-2)
  const double zsrc = two ? sec_bytes(a.gc, a.wc2.s.W) + tmp_bytes(LV(ctx, L - 2).g) : (o.has_z ? tmp_bytes(a.gc) : 0);
  double bytes = (a.has_y ? sec_bytes(v.g, a.Wy) : 0) + sec_bytes(v.g, a.rc.W) +
                 zsrc + (o.write_y ? sec_bytes(v.g, a.Wy) : 0) +
                 (o.corr ? 2 * sec_bytes(v.g, a.u_out.W) : 0) + (o.write_w ? tmp_bytes(v.g) : 0) +
                 (o.write_uh ? tmp_bytes(v.g) + tmp_bytes(a.gc) : 0);
  if (ctx->P.arith == CMG_ARITH_FP32)  // binary32 w: half the bytes
    bytes -= 0.5 * ((o.has_z ? tmp_bytes(a.gc) : 0) + (o.write_w ? tmp_bytes(v.g) : 0));
  bool fast = false;
  if (ctx->P.arith == CMG_ARITH_EXACT && ctx->fast && ctx->fb_tiles) {
    a.tiles = ctx->fb_tiles;
    if ((s = fb_slot(ctx, l, &a.ntiles))) return s;
  }
  ev_begin(ctx, kstat(ctx, CMG_KIND_SWEEP, l));
  if (ctx->P.arith != CMG_ARITH_EXACT) launch_sweep_fp(d, ctx->P.arith == CMG_ARITH_FP64, a, ctx->st);
  else if (!(fast = a.tiles && launch_sweep_fast(a, ctx->st))) launch_sweep(d, a, ctx->st);
  ev_end(ctx, kstat(ctx, CMG_KIND_SWEEP, l), bytes);
  if (fast) {
    ctx->launches++;  // the generic kernel over the fallback tiles
    ctx->fast_ctas += tiles_of(v.g);
    if (l == ctx->P.L_max) ctx->fast_ctas_top += tiles_of(v.g);
  }
  if ((s = launched(ctx, bytes))) return s;
  if (o.write_y) {
    v.ycur = 1 - v.ycur;
    v.y_zero = false;
  }
  return CMG_OK;
}

static cmg_status do_restrict(cmg_ctx *ctx, int l, bool first_sweep_below) {
  const int L = ctx->L, d = ctx->P.dim;
  Level &v = LV(ctx, l), &c = LV(ctx, l - 1);
  RestrictArgs a{};
  a.g = v.g;
  a.gc = c.g;
  a.has_y = !v.y_zero;
  a.y = sec_of(v.y[v.ycur]);
  a.rc = sec_of(rc_of(ctx, l));
  {
    cmg_status s1 = fresh_tmp_meta(ctx, c.accmeta);
    if (s1) return s1;
  }
  a.acc = tmp_of(c.acc, nullptr, c.accmeta);
  a.err = ctx->err;
  if (ctx->P.coef == CMG_COEF_DIFFUSION) {
    // d = fl(rc - A y~) in the cycle's type on level l, then rc_(l-1) = round(R d) in R's order
    a.d_out = ctx->dbuf;
    a.kfield = ctx->kfield;
    a.kN = (1 << ctx->P.L_max) + 1;
    a.kstride = 1 << (ctx->P.L_max - l);
    const double es = ctx->P.arith == CMG_ARITH_FP64 ? 8.0 : 4.0;  // d written, then read by the gather
    const double bytes = sec_bytes(v.g, a.y.W) + sec_bytes(v.g, a.rc.W) + 2 * es * v.g.nz * v.g.n * v.g.n;
    ev_begin(ctx, kstat(ctx, CMG_KIND_RESTRICT, l));
    launch_dvec_diffusion(d, ctx->P.arith == CMG_ARITH_FP64, a, ctx->st);
    GatherArgs ga{};
    ga.g = v.g;
    ga.gc = c.g;
    ga.d = ctx->dbuf;
    c.rc.W = Wr(ctx, l - 1, L);
    cmg_status s2 = fresh_meta(ctx, c.rc);
    if (s2) return s2;
    ga.rc_out = sec_of(c.rc);
    ga.err = ctx->err;
    launch_gather_restrict_fp(d, ctx->P.arith == CMG_ARITH_FP64, ga, ctx->st);
    ev_end(ctx, kstat(ctx, CMG_KIND_RESTRICT, l), bytes + sec_bytes(c.g, c.rc.W));
    LV(ctx, l - 1).y_zero = true;
    return launched(ctx, bytes + sec_bytes(c.g, c.rc.W));
  }
  ev_begin(ctx, kstat(ctx, CMG_KIND_RESTRICT, l));
  if (ctx->P.arith != CMG_ARITH_EXACT) launch_restrict_fp(d, ctx->P.arith == CMG_ARITH_FP64, a, ctx->st);
  else launch_restrict(d, a, ctx->st);
  ev_end(ctx, kstat(ctx, CMG_KIND_RESTRICT, l), sec_bytes(v.g, a.y.W) + sec_bytes(v.g, a.rc.W) + 2 * tmp_bytes(c.g));
  cmg_status s = launched(ctx, sec_bytes(v.g, a.y.W) + sec_bytes(v.g, a.rc.W) + 2 * tmp_bytes(c.g));
  if (s) return s;
  AccArgs b{};
  b.g = c.g;
  b.acc = tmp_of(c.acc, nullptr, c.accmeta);
  c.rc.W = Wr(ctx, l - 1, L);
  if ((s = fresh_meta(ctx, c.rc))) return s;
  b.r_out = sec_of(c.rc);
  b.first_sweep = first_sweep_below;
  if (first_sweep_below) {
    SecBuf &y = c.y[0];
    y.W = Wr(ctx, l - 1, L);
    if ((s = fresh_meta(ctx, y))) return s;
    b.y_out = sec_of(y);
    c.ycur = 0;
    c.y_zero = false;
  }
  b.chain = 0;
  jacobi_factor(ctx, l - 1, b.c_num, b.c_exp, b.cbits);
  b.err = ctx->err;
  const double bb = 2 * tmp_bytes(c.g) + sec_bytes(c.g, c.rc.W) * (first_sweep_below ? 2 : 1);
  ev_begin(ctx, kstat(ctx, CMG_KIND_ACC_ENCODE, l));
  launch_acc_encode(d, b, ctx->st);
  ev_end(ctx, kstat(ctx, CMG_KIND_ACC_ENCODE, l), bb);
  return launched(ctx, bb);
}

static cmg_status do_coarse(cmg_ctx *ctx, bool start, bool corr) {
  Level &v = LV(ctx, 1);
  CoarseArgs a{};
  a.dim = ctx->P.dim;
  a.mode_start = start;
  a.err = ctx->err;
  cmg_status s;
  if (start) {
    a.f1 = rhs_level1(ctx);
    a.Gf1 = ctx->scale_exp + ctx->fsh - ctx->P.dim * 1;
    v.u.W = Wu(ctx, 1, 1);
    if ((s = fresh_meta(ctx, v.u))) return s;
    a.u_out = sec_of(v.u);
    a.uh_out = tmp_of(v.uh, v.uhg, nullptr);
  } else {
    a.rc = sec_of(rc_of(ctx, 1));
    SecBuf &y = v.y[0];
    y.W = Wr(ctx, 1, ctx->L);
    if ((s = fresh_meta(ctx, y))) return s;
    a.y_out = sec_of(y);
    v.ycur = 0;
    v.y_zero = false;
    a.corr = corr;
    if (corr) {
      a.u_in = sec_of(v.u);
      SecBuf &ua = v.u_alt;  // level 1 < L_max here, so the spare buffer exists
      ua.W = Wu(ctx, 1, ctx->L);
      if ((s = fresh_meta(ctx, ua))) return s;
      a.u_out = sec_of(ua);
    }
    a.w_out = tmp_of(v.w, v.wg, nullptr);
    if (ctx->P.arith != CMG_ARITH_EXACT) {
      a.w_out_r = v.w;
      a.w_f64 = ctx->P.arith == CMG_ARITH_FP64;
    }
    if (corr) a.uh_out = tmp_of(v.uh, v.uhg, nullptr);
  }
  if (ctx->P.coef == CMG_COEF_DIFFUSION) {
    if (!ctx->kfield) return fail(ctx, CMG_EINVAL, "diffusion without a coefficient (cmg_set_coefficient)");
    a.kfield = ctx->kfield;
    a.kN = (1 << ctx->P.L_max) + 1;
    a.kstride = 1 << (ctx->P.L_max - 1);
    if (ctx->grhs) {  // the level-1 node is the centre of the finest grid
      const long long n1 = (1ll << ctx->P.L_max) - 1, c = n1 / 2;
      a.grhs = ctx->grhs;
      a.grhs_log2 = ctx->grhs_log2;
      a.gidx = ctx->P.dim == 3 ? (c * n1 + c) * n1 + c : c * n1 + c;
    }
  }
  ev_begin(ctx, kstat(ctx, CMG_KIND_COARSE, 1));
  launch_coarse(a, ctx->st);
  ev_end(ctx, kstat(ctx, CMG_KIND_COARSE, 1), 64);
  if ((s = launched(ctx, 64))) return s;
  if (!start && corr) std::swap(v.u, v.u_alt);
  return CMG_OK;
}

// ---------------------------------------------------------------- steps
static cmg_status need(cmg_ctx *ctx, bool cond, const char *what) {
  return cond ? CMG_OK : fail(ctx, CMG_EINVAL, "%s", what);
}

static cmg_status start_impl(cmg_ctx *ctx) {
  cmg_status s = need(ctx, ctx->have_rhs, "no right-hand side set");
  if (s) return s;
  ctx->meta_next = 1;
  CU(cudaMemsetAsync(ctx->meta_pool + 2 * ctx->meta_next, 0,
                     (size_t)(META_CAP - 2 * ctx->meta_next) * sizeof(int), ctx->st));
  if (ctx->fb_counts) {
    CU(cudaMemsetAsync(ctx->fb_counts, 0, FB_SLOTS * sizeof(int), ctx->st));
    ctx->fb_next = 0;
  }
  ctx->fast_ctas = ctx->fast_ctas_top = ctx->fb_done = ctx->fb_done_top = 0;
  CU(cudaMemsetAsync(ctx->err, 0, 8 * sizeof(int), ctx->st));
  for (int l = 1; l <= ctx->P.L_max; l++) {
    Level &v = LV(ctx, l);
    v.u.meta = v.r.meta = v.rc.meta = v.y[0].meta = v.y[1].meta = ctx->meta_pool;
    v.y_zero = true;
  }
  ctx->L = 1;
  s = do_coarse(ctx, true, false);
  ctx->uh_upto = 1;
  return s;
}

extern "C" cmg_status cmg_start(cmg_ctx *ctx) {
  if (!ctx) return CMG_EINVAL;
  graph_touch(ctx);
  return start_impl(ctx);
}

static cmg_status prolongate_impl(cmg_ctx *ctx) {
  cmg_status s = need(ctx, ctx->L >= 1 && ctx->L < ctx->P.L_max, "cannot prolongate at this level");
  if (s) return s;
  const int L = ctx->L + 1;
  // widen every coarser section by k_u bits (exact: appended zero bits)
  for (int l = 1; l < L; l++) {
    Level &v = LV(ctx, l);
    int Wn = Wu(ctx, l, L);
    if (Wn == v.u.W) continue;
    RepackArgs a{};
    a.in = sec_of(v.u);
    v.u_alt.W = Wn;
    if ((s = fresh_meta(ctx, v.u_alt))) return s;
    a.out = sec_of(v.u_alt);
    a.nblocks = v.g.nblocks;
    ev_begin(ctx, kstat(ctx, CMG_KIND_REPACK, l));
    launch_repack(a, ctx->st);
    ev_end(ctx, kstat(ctx, CMG_KIND_REPACK, l), sec_bytes(v.g, v.u.W) + sec_bytes(v.g, Wn));
    if ((s = launched(ctx, sec_bytes(v.g, v.u.W) + sec_bytes(v.g, Wn)))) return s;
    std::swap(v.u, v.u_alt);
  }
  Level &f = LV(ctx, L);
  if ((s = set_zero_section(ctx, f.u, f.g, Wu(ctx, L, L)))) return s;
  ctx->L = L;
  for (int l = 1; l <= L; l++) LV(ctx, l).y_zero = true;
  // u^_l for l < L keep their values (widening does not change values)
  return CMG_OK;
}

extern "C" cmg_status cmg_prolongate(cmg_ctx *ctx) {
  if (!ctx) return CMG_EINVAL;
  graph_touch(ctx);
  return prolongate_impl(ctx);
}

extern "C" cmg_status cmg_residual(cmg_ctx *ctx) {
  if (!ctx || ctx->L < 1) return CMG_EINVAL;
  graph_touch(ctx);
  return do_residual(ctx, false);
}

extern "C" cmg_status cmg_down(cmg_ctx *ctx, int l) {
  if (!ctx) return CMG_EINVAL;
  graph_touch(ctx);
  cmg_status s = need(ctx, l >= 2 && l <= ctx->L, "bad level");
  if (s) return s;
  Level &v = LV(ctx, l);
  v.y_zero = true;
  for (int k = 0; k < ctx->P.nu1; k++) {
    SweepOpts o;
    if ((s = do_sweep(ctx, l, o))) return s;
  }
  if (ctx->P.nu1 > 0) return do_restrict(ctx, l, false);
  return CMG_OK;  // rc_(l-1) = r_(l-1) from the residual chain
}

extern "C" cmg_status cmg_coarse(cmg_ctx *ctx) {
  if (!ctx || ctx->L < 1) return CMG_EINVAL;
  graph_touch(ctx);
  if (ctx->P.L_max == 1) return fail(ctx, CMG_EUNSUPPORTED, "cycle on a one-level hierarchy");
  return do_coarse(ctx, false, false);
}

// one post-smoothing sweep with the options o of its last launch: a Jacobi sweep,
// or a red half-sweep (y~ stored) followed by a black half-sweep carrying o
static cmg_status post_sweep(cmg_ctx *ctx, int l, SweepOpts o) {
  if (ctx->P.smoother != CMG_SMOOTHER_RBGS) return do_sweep(ctx, l, o);
  SweepOpts red;
  red.has_z = o.has_z;
  red.rb = 1;
  cmg_status s = do_sweep(ctx, l, red);
  if (s) return s;
  o.rb = 2;
  return do_sweep(ctx, l, o);
}

extern "C" cmg_status cmg_smooth(cmg_ctx *ctx, int l, int sweeps, int with_z) {
  if (!ctx) return CMG_EINVAL;
  graph_touch(ctx);
  cmg_status s = need(ctx, l >= 2 && l <= ctx->L && sweeps >= 0 && (with_z == 0 || with_z == 1),
                      "bad level, sweep count or with_z");
  if (s) return s;
  if (!with_z) {  // pre-smoothing: from y~_l = 0 while the coarser corrections are zero
    if (ctx->P.smoother != CMG_SMOOTHER_JACOBI)
      return fail(ctx, CMG_EUNSUPPORTED, "red-black Gauss-Seidel smooths on the up-leg only (nu1 = 0)");
    LV(ctx, l).y_zero = true;
    for (int k = 0; k < sweeps; k++) {
      SweepOpts o;
      if ((s = do_sweep(ctx, l, o))) return s;
    }
    return CMG_OK;
  }
  for (int k = 0; k < sweeps; k++) {  // post-smoothing with z_l = P_l w_(l-1); the last sweep writes w_l
    SweepOpts o;                        // for the next finer level of this FMG level
    o.has_z = true;
    o.write_w = (k == sweeps - 1) && l < ctx->L;
    if ((s = post_sweep(ctx, l, o))) return s;
  }
  return CMG_OK;
}

extern "C" cmg_status cmg_restrict(cmg_ctx *ctx, int l) {
  if (!ctx) return CMG_EINVAL;
  graph_touch(ctx);
  cmg_status s = need(ctx, l >= 2 && l <= ctx->L, "bad level");
  if (s) return s;
  if (ctx->P.nu1 == 0)
    return fail(ctx, CMG_EUNSUPPORTED, "without pre-smoothing the residual's restriction chain forms rc (Algorithm 2)");
  return do_restrict(ctx, l, false);
}

extern "C" cmg_status cmg_up(cmg_ctx *ctx, int l) {
  if (!ctx) return CMG_EINVAL;
  graph_touch(ctx);
  cmg_status s = need(ctx, l >= 2 && l <= ctx->L, "bad level");
  if (s) return s;
  for (int k = 0; k < ctx->P.nu2; k++) {
    SweepOpts o;
    o.has_z = true;
    o.write_w = (k == ctx->P.nu2 - 1) && l < ctx->L;  // w_l feeds the next finer level only
    if ((s = post_sweep(ctx, l, o))) return s;
  }
  return CMG_OK;
}

extern "C" cmg_status cmg_correct(cmg_ctx *ctx) {
  if (!ctx || ctx->L < 1) return CMG_EINVAL;
  graph_touch(ctx);
  cmg_status s;
  for (int l = 1; l <= ctx->L; l++) {
    Level &v = LV(ctx, l);
    if (v.y_zero) continue;
    AxpyArgs a{};
    a.g = v.g;
    a.u_in = sec_of(v.u);
    a.y = sec_of(v.y[v.ycur]);
    SecBuf un = v.u;  // in place
    un.W = Wu(ctx, l, ctx->L);
    if ((s = fresh_meta(ctx, un))) return s;
    a.u_out = sec_of(un);
    a.err = ctx->err;
    launch_axpy(a, ctx->st);
    if ((s = launched(ctx, 2 * sec_bytes(v.g, un.W) + sec_bytes(v.g, a.y.W)))) return s;
    v.u.meta = un.meta;
  }
  ctx->uh_upto = 0;
  return CMG_OK;
}

extern "C" cmg_status cmg_vcycle(cmg_ctx *ctx) {
  if (!ctx || ctx->L < 1) return CMG_EINVAL;
  graph_touch(ctx);
  cmg_status s = CMG_OK;
  for (int l = ctx->L; l >= 2 && !s; l--) s = cmg_down(ctx, l);
  if (!s) s = cmg_coarse(ctx);
  for (int l = 2; l <= ctx->L && !s; l++) s = cmg_up(ctx, l);
  return s;
}

// u^_L is written by the last IR iteration of an FMG level when the next level
// reads it materialized (not on the two-level path into L_max)
static bool need_uh_top(const cmg_ctx *ctx) {
  return ctx->L < ctx->P.L_max && !(ctx->tl && ctx->L == ctx->P.L_max - 1);
}

// the production IR iteration: residual with the first sweep fused, restriction
// with the next level's first sweep fused, corrections fused into the last up
// sweep of every level, u^ refreshed on the way up.
static cmg_status ir_fused(cmg_ctx *ctx, bool need_uh_top) {
  const int L = ctx->L, nu1 = ctx->P.nu1, nu2 = ctx->P.nu2;
  cmg_status s = do_residual(ctx, nu1 >= 1);
  if (s) return s;
  for (int l = L; l >= 2; l--) {
    Level &v = LV(ctx, l);
    if (nu1 == 0) {
      v.y_zero = true;
      continue;
    }
    const bool diff = ctx->P.coef == CMG_COEF_DIFFUSION;  // first sweeps not fused
    if (diff) v.y_zero = true;
    for (int k = diff ? 0 : 1; k < nu1; k++) {
      SweepOpts o;
      if ((s = do_sweep(ctx, l, o))) return s;
    }
    if ((s = do_restrict(ctx, l, !diff && l - 1 >= 2))) return s;
  }
  if ((s = do_coarse(ctx, false, true))) return s;
  for (int l = 2; l <= L; l++) {
    for (int k = 0; k < nu2; k++) {
      const bool last = (k == nu2 - 1);
      SweepOpts o;
      o.has_z = true;
      o.write_y = !last;
      o.corr = last;
      o.write_w = last && l < L;
      o.write_uh = last && (l < L || need_uh_top) && l < ctx->P.L_max;
      if ((s = post_sweep(ctx, l, o))) return s;
    }
  }
  // (on the two-level path level L - 1 keeps no u^: it is formed on the fly)
  ctx->uh_upto = tl_on(ctx) ? L - 2 : (need_uh_top && L < ctx->P.L_max) ? L : L - 1;
  return CMG_OK;
}

extern "C" cmg_status cmg_ir_iteration(cmg_ctx *ctx) {
  if (!ctx || ctx->L < 2) return ctx ? fail(ctx, CMG_EINVAL, "IR needs L >= 2") : CMG_EINVAL;
  graph_touch(ctx);
  return ir_fused(ctx, need_uh_top(ctx));
}

extern "C" cmg_status cmg_sync(cmg_ctx *ctx) {
  if (!ctx) return CMG_EINVAL;
  CU(cudaStreamSynchronize(ctx->st));
  int e[8] = {0};
  CU(cudaMemcpy(e, ctx->err, sizeof e, cudaMemcpyDeviceToHost));
  if (e[0] & ERR_CORRUPT) return fail(ctx, CMG_ECORRUPT, "invalid BFP code");
  if (e[0] & ERR_EXP) return fail(ctx, CMG_ERANGE, "block exponent outside [-127, 127]");
  if (e[0] & ERR_RANGE)
    return fail(ctx, CMG_ERANGE, "exact integer range exceeds 62 bits (site %d: |v| < 2^%d on grid 2^%d)", e[1], e[2],
                e[3]);
  return CMG_OK;
}

// Algorithm 3: the FMG levels, each with N_ir iterations of refinement
static cmg_status solve_body(cmg_ctx *ctx) {
  cmg_status s = start_impl(ctx);
  for (int L = 2; L <= ctx->P.L_max && !s; L++) {
    s = prolongate_impl(ctx);
    for (int it = 0; it < ctx->P.N_ir && !s; it++) s = ir_fused(ctx, it == ctx->P.N_ir - 1 && need_uh_top(ctx));
  }
  return s;
}

// Captures the solve into a graph and launches it.  Where the capture fails (a
// call that cannot be captured, such as the synchronisation of an overflowing
// fallback-count pool), nothing of it has run: the solve runs eagerly, and these
// inputs are not captured again.
static cmg_status graph_capture(cmg_ctx *ctx) {
  SolveGraph &gr = ctx->gr;
  CU(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeRelaxed));
  gr.capturing = true;
  cmg_status s = solve_body(ctx);
  gr.capturing = false;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->st, &graph);
  cudaGraphExec_t exec = nullptr;
  if (!s && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (s || e != cudaSuccess) {
    for (int k = 0; k < CMG_KIND_COUNT; k++) {  // events of the capture, never recorded
      for (int t = 0; t < 2; t++) {
        for (auto &p : ctx->stats[k][t].ev) {
          cudaEventDestroy(p.first);
          cudaEventDestroy(p.second);
        }
        ctx->stats[k][t].ev.clear();
        ctx->stats[k][t].bytes = 0;
        ctx->stats[k][t].launches = 0;
      }
    }
    cudaGetLastError();
    ctx->launches = 0;
    ctx->alg_bytes = 0;
    gr.failed = true;
    return solve_body(ctx);  // also reports any error of the host logic itself
  }
  gr.exec = exec;
  gr.captures++;
  graph_save(ctx);
  CU(cudaGraphLaunch(exec, ctx->st));
  gr.graph_solves++;
  return CMG_OK;
}

extern "C" cmg_status cmg_fmg_solve(cmg_ctx *ctx, cmg_report *rep) {
  if (!ctx) return CMG_EINVAL;
  for (int k = 0; k < CMG_KIND_COUNT; k++) {
    stat_reset(ctx->stats[k][0]);
    stat_reset(ctx->stats[k][1]);
  }
  ctx->launches = 0;
  ctx->alg_bytes = 0;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0, ctx->st));
  // the first solve of new inputs runs eagerly, the second is captured, later
  // ones launch the graph
  cmg_status s = CMG_OK;
  const bool usable = graph_usable(ctx);
  if (usable && ctx->gr.exec) {
    graph_restore(ctx);
    CU(cudaGraphLaunch(ctx->gr.exec, ctx->st));
    ctx->gr.graph_solves++;
  } else if (usable && ctx->gr.warm > 0) {
    s = graph_capture(ctx);
  } else {
    s = solve_body(ctx);
    if (!s && usable) ctx->gr.warm++;
  }
  CU(cudaEventRecord(e1, ctx->st));
  cmg_status s2 = cmg_sync(ctx);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  if (s2) return s2;
  if (rep) {
    std::memset(rep, 0, sizeof *rep);
    const int d = ctx->P.dim, Lm = ctx->P.L_max;
    rep->solve_ms = ms;
    rep->dofs = (int64_t)make_geo(d, Lm).nz * make_geo(d, Lm).n * make_geo(d, Lm).n;
    rep->launches = ctx->launches;
    rep->alg_bytes = ctx->alg_bytes;
    double bits = 0, tb = 0;
    for (int l = 1; l <= Lm; l++) {
      Geo g = make_geo(d, l);
      bits += (double)g.nblocks * (32.0 * (Wu(ctx, l, Lm) + 3 * Wr(ctx, l, Lm)) + 8.0 * 4);
      // u^, w and the restriction accumulator (two-level path: level L_max - 1 only the last)
      if (l < Lm) tb += (ctx->tl && l == Lm - 1 ? 1.0 : 3.0) * 8.0 * g.nz * g.n * g.R;
      // without pre-smoothing: the restriction chain's t^ section on every level
      if (ctx->P.nu1 == 0 && l < Lm) tb += (double)g.nblocks * (4.0 * (ctx->P.k_u * Lm + ctx->P.b1) + 1.0);
    }
    rep->persistent_bits = bits;
    rep->temp_bytes = tb;
    for (int k = 0; k < CMG_KIND_COUNT; k++) {
      ev_collect(ctx->stats[k][0]);
      ev_collect(ctx->stats[k][1]);
    }
    const KStat &sw = ctx->stats[CMG_KIND_SWEEP][1], &rs = ctx->stats[CMG_KIND_RESIDUAL][1];
    rep->sweep_ms_total = sw.ms;
    rep->sweep_launches = sw.launches;
    rep->sweep_alg_bytes = sw.bytes;
    rep->resid_ms_total = rs.ms;
    rep->resid_launches = rs.launches;
    rep->resid_alg_bytes = rs.bytes;
  }
  return CMG_OK;
}

extern "C" cmg_status cmg_kernel_stats(cmg_ctx *ctx, int kind, int top, double *ms, int64_t *launches,
                                       double *bytes) {
  if (!ctx || kind < 0 || kind >= CMG_KIND_COUNT || top < 0 || top > 1) return CMG_EINVAL;
  KStat &k = ctx->stats[kind][top];
  ev_collect(k);
  if (ms) *ms = k.ms;
  if (launches) *launches = k.launches;
  if (bytes) *bytes = k.bytes;
  return CMG_OK;
}

// ---------------------------------------------------------------- section access
static SecBuf *pick(cmg_ctx *ctx, int which, int l) {
  Level &v = LV(ctx, l);
  switch (which) {
    case CMG_SEC_U: return &v.u;
    case CMG_SEC_R: return &v.r;
    case CMG_SEC_RC: return &rc_of(ctx, l);
    case CMG_SEC_Y: return &v.y[v.ycur];
  }
  return nullptr;
}

extern "C" int cmg_section_width(const cmg_ctx *ctx, int which, int level) {
  if (!ctx || level < 1 || level > ctx->P.L_max) return -1;
  int L = ctx->L < level ? level : ctx->L;
  return which == CMG_SEC_U ? Wu(ctx, level, L) : Wr(ctx, level, L);
}

// Device bytes into host memory.  Page-locked memory the GPU maps (the whole
// range: both ends are checked) is written by a copy kernel through that
// mapping on the context's stream; other host memory, or an unaligned buffer,
// by cudaMemcpy.  The DMA copy of a large section straight after a solve ran at
// a fraction of the link's rate on GB300, the kernel at the full rate.
static cmg_status copy_out(cmg_ctx *ctx, void *dst, const void *src, size_t bytes) {
  if (!bytes) return CMG_OK;
  cudaPointerAttributes a0{}, a1{};
  const bool mapped = cudaPointerGetAttributes(&a0, dst) == cudaSuccess && a0.type == cudaMemoryTypeHost &&
                      a0.devicePointer &&
                      cudaPointerGetAttributes(&a1, (const char *)dst + bytes - 1) == cudaSuccess &&
                      a1.type == cudaMemoryTypeHost &&
                      (const char *)a1.devicePointer == (const char *)a0.devicePointer + bytes - 1;
  cudaGetLastError();  // an unregistered pointer is not an error here
  if (mapped && ((uintptr_t)a0.devicePointer % 16) == 0 && ((uintptr_t)src % 16) == 0) {
    int dev = 0, nsm = 1;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    launch_copy_out(src, a0.devicePointer, bytes, nsm, ctx->st);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(ctx->st));
    return CMG_OK;
  }
  CU(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
  return CMG_OK;
}

extern "C" cmg_status cmg_get_section(cmg_ctx *ctx, int which, int level, uint32_t *words, int8_t *exps) {
  if (!ctx || level < 1 || level > ctx->L || !exps) return CMG_EINVAL;
  SecBuf *b = pick(ctx, which, level);
  if (!b) return CMG_EINVAL;
  cmg_status s = cmg_sync(ctx);
  if (s) return s;
  const Geo &g = LV(ctx, level).g;
  if (which == CMG_SEC_Y && LV(ctx, level).y_zero) {
    std::memset(exps, 0x80, (size_t)g.nblocks);
    if (words) std::memset(words, 0, (size_t)g.nblocks * Wr(ctx, level, ctx->L) * 4);
    return CMG_OK;
  }
  cmg_status s2 = copy_out(ctx, exps, b->exps, (size_t)g.nblocks);
  if (!s2 && words) s2 = copy_out(ctx, words, b->words, (size_t)g.nblocks * b->W * 4);
  return s2;
}

extern "C" cmg_status cmg_set_section(cmg_ctx *ctx, int which, int level, int W, const uint32_t *words,
                                      const int8_t *exps) {
  if (!ctx || level < 1 || level > ctx->L || !words || !exps || W < 2 || W > 32) return CMG_EINVAL;
  graph_touch(ctx);
  SecBuf *b = pick(ctx, which, level);
  if (!b) return CMG_EINVAL;
  const Geo &g = LV(ctx, level).g;
  if ((size_t)g.nblocks * W > b->cap_words) return fail(ctx, CMG_EINVAL, "width above the allocated width");
  int emax = 0, eminn = 0;
  for (long long i = 0; i < g.nblocks; i++)
    if (exps[i] != -128) {
      emax = std::max(emax, exps[i] + META_BIAS);
      eminn = std::max(eminn, META_BIAS - exps[i]);
    }
  cmg_status s = fresh_meta(ctx, *b);
  if (s) return s;
  int m[2] = {emax, eminn};
  CU(cudaStreamSynchronize(ctx->st));
  CU(cudaMemcpy(b->meta, m, sizeof m, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(b->exps, exps, (size_t)g.nblocks, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(b->words, words, (size_t)g.nblocks * W * 4, cudaMemcpyHostToDevice));
  b->W = W;
  if (which == CMG_SEC_Y) LV(ctx, level).y_zero = false;
  if (which == CMG_SEC_U) ctx->uh_upto = std::min(ctx->uh_upto, level - 1);
  return CMG_OK;
}

extern "C" cmg_status cmg_decode_solution(cmg_ctx *ctx, int64_t z0, int64_t nz, double *out) {
  if (!ctx || !out || ctx->L < 1) return CMG_EINVAL;
  const int L = ctx->L;
  const Geo &g = LV(ctx, L).g;
  if (z0 < 0 || nz < 0 || z0 + nz > g.nz) return CMG_EINVAL;
  cmg_status s;
  const bool two = tl_on(ctx);  // u^_(L-1) = u~_(L-1) + P u^_(L-2) on the fly
  const int need = two ? L - 2 : L - 1;
  if (ctx->uh_upto < need) {
    if ((s = run_chain(ctx, need))) return s;
    ctx->uh_upto = need;
  }
  DecodeSolArgs a{};
  a.g = g;
  a.gc = L > 1 ? LV(ctx, L - 1).g : g;
  a.u = sec_of(LV(ctx, L).u);
  a.has_uhc = L > 1;
  if (two) {
    a.tl = 1;
    a.uhc2 = two_level(ctx, LV(ctx, L - 1).u, false);
  } else if (L > 1) {
    a.uhc = tmp_of(LV(ctx, L - 1).uh, LV(ctx, L - 1).uhg, nullptr);
  }
  a.z0 = z0;
  a.nz = nz;
  a.out = out;
  a.err = ctx->err;
  launch_decode_solution(ctx->P.dim, a, ctx->st);
  if ((s = launched(ctx, 0))) return s;
  return cmg_sync(ctx);
}

// ---------------------------------------------------------------- checkpoint
struct StateHeader {
  char magic[8];
  cmg_params P;
  int L;
};

extern "C" cmg_status cmg_state_save(cmg_ctx *ctx, void *buf, size_t *len) {
  if (!ctx || !len || ctx->L < 1) return CMG_EINVAL;
  size_t need_b = sizeof(StateHeader);
  for (int l = 1; l <= ctx->L; l++) {
    const Geo &g = LV(ctx, l).g;
    need_b += sizeof(int) + (size_t)g.nblocks + (size_t)g.nblocks * LV(ctx, l).u.W * 4;
  }
  if (!buf) {
    *len = need_b;
    return CMG_OK;
  }
  if (*len < need_b) return fail(ctx, CMG_EINVAL, "buffer too small");
  cmg_status s = cmg_sync(ctx);
  if (s) return s;
  char *p = (char *)buf;
  StateHeader h;
  std::memcpy(h.magic, "CMGSTAT1", 8);
  h.P = ctx->P;
  h.L = ctx->L;
  std::memcpy(p, &h, sizeof h);
  p += sizeof h;
  for (int l = 1; l <= ctx->L; l++) {
    const SecBuf &u = LV(ctx, l).u;
    const Geo &g = LV(ctx, l).g;
    std::memcpy(p, &u.W, sizeof(int));
    p += sizeof(int);
    CU(cudaMemcpy(p, u.exps, (size_t)g.nblocks, cudaMemcpyDeviceToHost));
    p += g.nblocks;
    CU(cudaMemcpy(p, u.words, (size_t)g.nblocks * u.W * 4, cudaMemcpyDeviceToHost));
    p += (size_t)g.nblocks * u.W * 4;
  }
  *len = need_b;
  return CMG_OK;
}

extern "C" cmg_status cmg_state_load(cmg_ctx *ctx, const void *buf, size_t len) {
  if (!ctx || !buf || len < sizeof(StateHeader)) return CMG_EINVAL;
  graph_touch(ctx);
  StateHeader h;
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, "CMGSTAT1", 8) || std::memcmp(&h.P, &ctx->P, sizeof h.P) || h.L < 1 ||
      h.L > ctx->P.L_max)
    return fail(ctx, CMG_EINVAL, "checkpoint does not match this context");
  const char *p = (const char *)buf + sizeof h;
  size_t left = len - sizeof h;
  ctx->L = h.L;
  for (int l = 1; l <= h.L; l++) {
    const Geo &g = LV(ctx, l).g;
    int W;
    if (left < sizeof(int)) return fail(ctx, CMG_EINVAL, "truncated checkpoint");
    std::memcpy(&W, p, sizeof W);
    size_t need_b = sizeof(int) + (size_t)g.nblocks + (size_t)g.nblocks * W * 4;
    if (W < 2 || W > 32 || left < need_b) return fail(ctx, CMG_EINVAL, "truncated checkpoint");
    const int8_t *e = (const int8_t *)(p + sizeof(int));
    const uint32_t *w = (const uint32_t *)(p + sizeof(int) + g.nblocks);
    std::vector<uint32_t> wtmp(w, w + (size_t)g.nblocks * W);  // alignment
    cmg_status s = cmg_set_section(ctx, CMG_SEC_U, l, W, wtmp.data(), e);
    if (s) return s;
    p += need_b;
    left -= need_b;
  }
  for (int l = 1; l <= h.L; l++) LV(ctx, l).y_zero = true;
  ctx->uh_upto = 0;
  return CMG_OK;
}

// ---------------------------------------------------------------- stand-alone codec
// The codec's error word: one per host thread and device, allocated on the
// thread's first codec call on that device and kept for the process (a codec
// call waits for its own work, so one host thread never has two calls in
// flight, and calls from different threads never share a word).
constexpr int CODEC_MAX_DEVICES = 64;
static thread_local int *t_codec_err[CODEC_MAX_DEVICES];

static cmg_status codec_err_word(int **out, cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= CODEC_MAX_DEVICES) return CMG_ECUDA;
  if (!t_codec_err[dev] && cudaMalloc(&t_codec_err[dev], sizeof(int)) != cudaSuccess) {
    t_codec_err[dev] = nullptr;
    return CMG_ENOMEM;
  }
  if (cudaMemsetAsync(t_codec_err[dev], 0, sizeof(int), st) != cudaSuccess) return CMG_ECUDA;
  *out = t_codec_err[dev];
  return CMG_OK;
}

static cmg_status codec_finish(int *err, cudaStream_t st) {
  int e = 0;
  if (cudaGetLastError() != cudaSuccess) return CMG_ECUDA;
  if (cudaMemcpyAsync(&e, err, sizeof e, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return CMG_ECUDA;
  if (e & ERR_INPUT) return CMG_EINVAL;
  if (e & ERR_CORRUPT) return CMG_ECORRUPT;
  if (e & ERR_EXP) return CMG_ERANGE;
  return CMG_OK;
}

extern "C" cmg_status cmg_encode(const double *x, int64_t n, int W, uint32_t *words, int8_t *exps, void *stream) {
  if (n < 0 || W < 2 || W > 32 || (n > 0 && (!x || !words || !exps))) return CMG_EINVAL;
  if (n == 0) return CMG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int *err = nullptr;
  cmg_status s = codec_err_word(&err, st);
  if (s != CMG_OK) return s;
  CodecArgs a{};
  a.x = const_cast<double *>(x);
  a.n = n;
  a.W = W;
  a.words = words;
  a.exps = exps;
  a.err = err;
  launch_encode_f64(a, st);
  return codec_finish(err, st);
}

extern "C" cmg_status cmg_decode(const uint32_t *words, const int8_t *exps, int64_t n, int W, double *x,
                                 void *stream) {
  if (n < 0 || W < 2 || W > 32 || (n > 0 && (!x || !words || !exps))) return CMG_EINVAL;
  if (n == 0) return CMG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int *err = nullptr;
  cmg_status s = codec_err_word(&err, st);
  if (s != CMG_OK) return s;
  CodecArgs a{};
  a.x = x;
  a.n = n;
  a.W = W;
  a.words = const_cast<uint32_t *>(words);
  a.exps = const_cast<int8_t *>(exps);
  a.err = err;
  launch_decode_f64(a, st);
  return codec_finish(err, st);
}

// ---------------------------------------------------------------- storage model
// Sec. 6.1.4 mantissa counts of CMG (regressive) and BFPMG (progressive) storage;
// see include/cmg.h for the formulas.
extern "C" cmg_status cmg_storage_model(int dim, int L, int k_u, int k_r, int b1, int b2, cmg_storage *out) {
  if (!out || dim < 1 || dim > 3 || L < 1 || L > 40 || k_u < 0 || k_r < 0 || b1 < 1 || b2 < 1)
    return CMG_EINVAL;
  auto n_of = [dim](int l) {
    if (l < 1) return 0.0;
    const double side = std::ldexp(1.0, l) - 1.0;
    double v = 1.0;
    for (int a = 0; a < dim; a++) v *= side;
    return v;
  };
  double cu = 0, cr = 0, py = 0;
  for (int l = 1; l <= L; l++) {
    const double n = n_of(l);
    cu += n * (double)(k_u * (L - l) + b1);
    cr += n * (double)(k_r * (L - l) + b2);
    py += n * (double)(k_r * (l - 1) + b2);
  }
  const double nL = n_of(L);
  cmg_storage s{};
  s.dofs = nL;
  s.cmg_vector_bits = cu;
  s.cmg_fmg_bits = cu + 2 * cr;
  s.bfpmg_vector_bits = nL * (double)(k_u * (L - 1) + b1);
  s.bfpmg_fmg_bits = s.bfpmg_vector_bits + nL * (double)(k_r * (L - 1) + b2) +
                     n_of(L - 1) * (double)(k_r * (L - 2) + b2) + py;
  s.vector_saving = s.bfpmg_vector_bits / s.cmg_vector_bits;
  s.fmg_saving = s.bfpmg_fmg_bits / s.cmg_fmg_bits;
  *out = s;
  return CMG_OK;
}
