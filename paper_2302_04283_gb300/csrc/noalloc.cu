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
  if (!ctx) return RAD_EINVAL;
  if (!ctx->have_metric) return fail(ctx, RAD_ESTATE, "rad_set_metric has not been called");
  if (!o || !gas) return fail(ctx, RAD_EINVAL, "null opts or gas");
  if (o->precision != RAD_F64 && o->precision != RAD_F32) return fail(ctx, RAD_EINVAL, "bad precision");
  if (o->recon != RAD_RECON_DC && o->recon != RAD_RECON_PLM) return fail(ctx, RAD_EINVAL, "bad recon");
  if (o->coupling < RAD_COUPLE_THERMAL || o->coupling > RAD_COUPLE_NONE) return fail(ctx, RAD_EINVAL, "bad coupling");
  if (o->coupling == RAD_COUPLE_THERMAL && !(o->gamma > 1.0)) return fail(ctx, RAD_EINVAL, "gamma must be > 1");
  if (!(o->n0crit >= 0.0)) return fail(ctx, RAD_EINVAL, "n0crit must be >= 0");
  if (o->coupling != RAD_COUPLE_NONE && (!gas->rho || !gas->u || !gas->alpha_a || !gas->alpha_s))
    return fail(ctx, RAD_EINVAL, "gas fields rho, u, alpha_a, alpha_s are required for coupling");
  if (o->coupling == RAD_COUPLE_EMISSIVITY && !gas->eta)
    return fail(ctx, RAD_EINVAL, "emissivity coupling needs gas->eta");
  if (!gas->T) return fail(ctx, RAD_EINVAL, "gas->T is required");
  if (!I || ((uintptr_t)I & 15u)) return fail(ctx, RAD_EINVAL, "I must be a 16-byte aligned device pointer");
  if (!(dt > 0.0) || !(dt < 1e300)) return fail(ctx, RAD_EINVAL, "dt must be finite and > 0");
  if (ctx->ang.n_ang > rad::kMaxBinsStep)
    return fail(ctx, RAD_EUNSUPPORTED, "rad_step_noalloc supports up to 812 bins (geodesic level 9)");
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
