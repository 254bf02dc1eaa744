// rad_step_noalloc: the RK2 step with its stage scratch in a static device
// array instead of memory from cudaMalloc.
//
// Who needs it: a caller whose device memory is owned by a host framework's
// pool and which must not make driver allocations after start-up, or a
// latency-bound loop that cannot afford the implicit device synchronisation
// cudaMalloc / cudaFree may perform.  rad_step allocates its scratch (one
// intensity array and one temperature array) on its first call and whenever
// the grid grows; this variant never allocates.
//
// The scratch is a file-scope static __device__ array of kNoAllocBytes.  Every
// GPU that loads the library holds it until the process exits, and every call
// of this entry point on a device shares it, so calls that overlap on the GPU
// (two streams, or two contexts on one device) race on it.  The array keeps
// the last call's contents; nothing in it has to start at zero, because the
// step writes every scratch element it later reads within the same call.
//
// In host code the array's name is only a host-side stand-in.  Its device
// address is looked up once per device, with that device current, by
// cudaGetSymbolAddress on the first call on that device; that first call
// should therefore come before any stream capture.
#include <mutex>

#include "rad_internal.h"

namespace {

constexpr size_t kNoAllocBytes = (size_t)32 << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_step_scratch[kNoAllocBytes];

std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

int scratch_address(void **out, std::string &err) {
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) {
    err = std::string("rad_step_noalloc: cudaGetDevice failed: ") + cudaGetErrorString(ce);
    return RAD_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    err = "rad_step_noalloc: device index out of range";
    return RAD_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    ce = cudaGetSymbolAddress(&p, g_step_scratch);
    if (ce != cudaSuccess || !p) {
      err = std::string("rad_step_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(ce);
      return RAD_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return RAD_OK;
}

int fail(rad_ctx *ctx, int code, const std::string &msg) {
  ctx->last_error = msg;
  return code;
}

}  // namespace

extern "C" int rad_step_noalloc(rad_ctx *ctx, void *I, const rad_gas *gas, double dt, const rad_opts *o,
                                double *gas_src) {
  // the same host-side checks as rad_step, before anything is launched
  const int chk = rad::check_step_args(ctx, I, gas, dt, o);
  if (chk != RAD_OK) return chk;
  if (ctx->n_groups > 0) return fail(ctx, RAD_EUNSUPPORTED, "rad_step_noalloc steps gray transport (no groups)");
  const rad::DevGeom &G = ctx->geom;
  const size_t ncell = (size_t)G.n[0] * G.n[1] * G.n[2];
  const size_t esz = o->precision == RAD_F32 ? 4 : 8;
  const size_t ibytes = (ncell * ctx->ang.n_ap * esz + 255) / 256 * 256;
  const size_t need = ibytes + ncell * sizeof(double);
  if (need > kNoAllocBytes)
    return fail(ctx, RAD_EINVAL,
                "rad_step_noalloc: the grid needs " + std::to_string(need) +
                    " bytes of stage scratch, more than the 33554432-byte static array; use rad_step");
  void *base = nullptr;
  std::string err;
  int st = scratch_address(&base, err);
  if (st != RAD_OK) return fail(ctx, st, err);
  double *scratch_T = (double *)((unsigned char *)base + ibytes);
  st = rad::launch_step(ctx, I, gas, dt, o, gas_src, base, scratch_T, err);
  return st == RAD_OK ? st : fail(ctx, st, err);
}
