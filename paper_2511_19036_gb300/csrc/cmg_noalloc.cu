// Decoding a compact vector without allocating device memory.
//
// cmg_decode_compact() turns the sections u~_1 .. u~_L of a compact vector into
// the standard representation u^_L (FP64) with the same kernels that
// cmg_decode_solution() uses.  Those kernels need scratch space for the decoded
// coarse levels u^_1 .. u^_(L-1) (int64 values with one grid per 32-value block)
// and for an error word.  cmg_decode_solution() takes that space from a solver
// context, which allocates it with cudaMalloc.  Here it lives in one file-scope
// __device__ array instead, so the call itself never allocates.
//
// This is for callers that must not allocate device memory during their run:
// for instance a host application that hands all of its device memory to its
// own pool allocator at start-up, or a latency-critical loop in which the
// implicit device-wide synchronisation of cudaMalloc/cudaFree cannot be
// tolerated.
//
// The price of the static array: every GPU that loads this library holds
// CMG_STATIC_SCRATCH_BYTES of device memory until the process exits, and all
// calls on a device share it (see include/cmg.h).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "../../include/cmg.h"
#include "cmg_device.cuh"
#include "cmg_kernels.h"

using namespace cmg;

namespace {

constexpr size_t SCRATCH_BYTES = CMG_STATIC_SCRATCH_BYTES;
constexpr size_t ERR_BYTES = 256;  // error word block, kept 256-byte aligned

// The scratch array.  Host code must not use its address directly (in host
// code the name is only a stand-in); the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// On every call, with the caller's device current: look up the array's device
// address.  The lookup is a host-side query and cheap; it is not cached, because
// a device reset (or a new primary context) reloads the module and moves the
// array, and a cached address would then be stale.
cmg_status scratch_for_current_device(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CMG_ECUDA;
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return CMG_ECUDA;
  *out = (unsigned char *)p;
  return CMG_OK;
}

Geo geo_of(int dim, int l) {
  Geo g;
  g.l = l;
  g.n = (1 << l) - 1;
  g.nz = dim == 3 ? g.n : 1;
  g.nbx = (g.n + 31) / 32;
  g.R = 32 * g.nbx;
  g.nblocks = (long long)g.nz * g.n * g.nbx;
  return g;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" size_t cmg_decode_compact_scratch_bytes(int dim, int L) {
  if ((dim != 2 && dim != 3) || L < 1 || L > 30) return (size_t)-1;
  size_t need = ERR_BYTES;
  for (int l = 1; l < L; l++) {
    Geo g = geo_of(dim, l);
    need += round256((size_t)g.nz * g.n * g.R * sizeof(long long));
    need += round256((size_t)g.nblocks * sizeof(int));
  }
  return need;
}

extern "C" cmg_status cmg_decode_compact(int dim, int L, const uint32_t *const *words_dev,
                                         const int8_t *const *exps_dev, const int *widths, int64_t z0,
                                         int64_t nz, double *out_dev, void *cuda_stream) {
  if ((dim != 2 && dim != 3) || L < 1 || L > 14 || !words_dev || !exps_dev || !widths || !out_dev)
    return CMG_EINVAL;
  for (int l = 0; l < L; l++)
    if (!words_dev[l] || !exps_dev[l] || widths[l] < 2 || widths[l] > 32) return CMG_EINVAL;
  const Geo top = geo_of(dim, L);
  if (z0 < 0 || nz < 0 || z0 + nz > top.nz) return CMG_EINVAL;
  // the coarse levels must fit the static array: refuse anything larger
  if (cmg_decode_compact_scratch_bytes(dim, L) > SCRATCH_BYTES) return CMG_ERANGE;
  if (nz == 0) return CMG_OK;

  unsigned char *base = nullptr;
  cmg_status s = scratch_for_current_device(&base);
  if (s != CMG_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int *err = (int *)base;
  // the array keeps the previous call's contents: the error words must start at 0
  if (cudaMemsetAsync(err, 0, ERR_BYTES, st) != cudaSuccess) return CMG_ECUDA;

  // carve u^_1 .. u^_(L-1) (values and block grids) out of the array; every
  // entry is written by the chain before it is read, so no clearing is needed
  unsigned char *p = base + ERR_BYTES;
  Tmp prev{};
  for (int l = 1; l < L; l++) {
    Geo g = geo_of(dim, l);
    Tmp cur{};
    cur.v = (long long *)p;
    p += round256((size_t)g.nz * g.n * g.R * sizeof(long long));
    cur.gb = (int *)p;
    p += round256((size_t)g.nblocks * sizeof(int));
    ChainArgs a{};
    a.g = g;
    a.gc = l > 1 ? geo_of(dim, l - 1) : g;
    a.u.words = const_cast<uint32_t *>(words_dev[l - 1]);
    a.u.exps = const_cast<int8_t *>(exps_dev[l - 1]);
    a.u.W = widths[l - 1];
    a.has_uhc = l > 1;
    a.uhc = prev;
    a.uh_out = cur;
    a.err = err;
    launch_chain(dim, a, st);
    if (cudaGetLastError() != cudaSuccess) return CMG_ECUDA;
    prev = cur;
  }
  DecodeSolArgs d{};
  d.g = top;
  d.gc = L > 1 ? geo_of(dim, L - 1) : top;
  d.u.words = const_cast<uint32_t *>(words_dev[L - 1]);
  d.u.exps = const_cast<int8_t *>(exps_dev[L - 1]);
  d.u.W = widths[L - 1];
  d.has_uhc = L > 1;
  d.uhc = prev;
  d.z0 = z0;
  d.nz = nz;
  d.out = out_dev;
  d.err = err;
  launch_decode_solution(dim, d, st);
  if (cudaGetLastError() != cudaSuccess) return CMG_ECUDA;
  int e[8];
  if (cudaMemcpyAsync(e, err, sizeof e, cudaMemcpyDeviceToHost, st) != cudaSuccess) return CMG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CMG_ECUDA;
  if (e[0] & ERR_CORRUPT) return CMG_ECORRUPT;
  if (e[0] & (ERR_EXP | ERR_RANGE)) return CMG_ERANGE;
  return CMG_OK;
}
