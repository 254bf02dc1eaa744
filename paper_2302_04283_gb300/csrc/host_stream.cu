// rad_step_host: the radiation step for data that lives in host memory.
//
// For each item the intensity and the gas state are copied to the device,
// advanced by rad_step, contracted by rad_moments, and the moments (plus the
// updated temperature and, on request, the intensity) are copied back.  Two
// device slots alternate: the copies of one item run on a second stream
// while the context stream computes the other, so that with pinned host
// buffers the transfer time hides behind the kernels.  The paper has no
// counterpart (it assumes the fields are resident).
//
// Order on the copy stream: H2D(0), then for every item i: H2D(i + 1) (after
// the compute of item i - 1 has released that slot), D2H(i) (after the
// compute of item i).  The context stream waits for H2D(i) and runs the steps
// of item i; a third stream runs its moment contraction, so that the
// (bandwidth-bound) contraction of one item overlaps the steps of the next.
#include <cstring>

#include "rad_internal.h"

namespace {

int fail_h(rad_ctx *ctx, int code, const std::string &msg) {
  ctx->last_error = msg;
  return code;
}

struct Slot {
  void *I = nullptr;
  double *rho = nullptr, *u = nullptr, *aa = nullptr, *as = nullptr, *eta = nullptr, *T = nullptr;
  void *R = nullptr;
};

}  // namespace

extern "C" int rad_step_host(rad_ctx *ctx, int n_items, const rad_host_item *items, double dt, const rad_opts *o,
                             int nsteps, int frame, int method) {
  if (!ctx) return RAD_EINVAL;
  if (!ctx->have_metric) return fail_h(ctx, RAD_ESTATE, "rad_set_metric has not been called");
  if (n_items < 0 || !o || nsteps < 1) return fail_h(ctx, RAD_EINVAL, "bad item count, options or step count");
  if (n_items == 0) return RAD_OK;
  if (!items) return fail_h(ctx, RAD_EINVAL, "null items");
  const bool f32 = o->precision == RAD_F32;
  if (!f32 && o->precision != RAD_F64) return fail_h(ctx, RAD_EINVAL, "bad precision");
  if (frame < RAD_FRAME_TETRAD || frame > RAD_FRAME_FLUID) return fail_h(ctx, RAD_EINVAL, "bad frame");
  if (method != RAD_MOM_SIMT && method != RAD_MOM_BF16X3) return fail_h(ctx, RAD_EINVAL, "bad method");
  if (method == RAD_MOM_BF16X3 && !f32) return fail_h(ctx, RAD_EINVAL, "the split-bf16 moments read float intensities");
  const bool with_eta = o->coupling == RAD_COUPLE_EMISSIVITY;
  for (int i = 0; i < n_items; ++i) {
    const rad_host_item &it = items[i];
    if (!it.I || !it.rho || !it.u || !it.alpha_a || !it.alpha_s || !it.T || !it.R || (with_eta && !it.eta))
      return fail_h(ctx, RAD_EINVAL, "rad_step_host: null host array in item " + std::to_string(i));
  }
  const rad::DevGeom &G = ctx->geom;
  const size_t ncell = (size_t)G.n[0] * G.n[1] * G.n[2];
  const size_t esz = f32 ? 4 : 8;
  const size_t bI = ncell * ctx->ang.n_ap * esz, bC = ncell * sizeof(double), bR = ncell * 10 * esz;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t per_slot = up(bI) + 6 * up(bC) + up(3 * bC) + up(bR);
  if (ctx->host_slot_bytes < 2 * per_slot) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->host_slot_buf);
    ctx->host_slot_buf = nullptr;
    ctx->host_slot_bytes = 0;
    if (cudaMalloc(&ctx->host_slot_buf, 2 * per_slot) != cudaSuccess)
      return fail_h(ctx, RAD_ENOMEM, "rad_step_host: slot allocation failed");
    ctx->host_slot_bytes = 2 * per_slot;
  }
  if (!ctx->copy_stream) {
    if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->mom_stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail_h(ctx, RAD_ECUDA, "rad_step_host: stream creation failed");
    for (int s = 0; s < 2; ++s) {
      cudaEventCreateWithFlags(&ctx->ev_h2d[s], cudaEventDisableTiming);
      cudaEventCreateWithFlags(&ctx->ev_step[s], cudaEventDisableTiming);
      cudaEventCreateWithFlags(&ctx->ev_done[s], cudaEventDisableTiming);
    }
  }
  Slot slot[2];
  for (int s = 0; s < 2; ++s) {
    unsigned char *p = (unsigned char *)ctx->host_slot_buf + s * per_slot;
    slot[s].I = p;
    p += up(bI);
    double **f[5] = {&slot[s].rho, &slot[s].aa, &slot[s].as, &slot[s].eta, &slot[s].T};
    for (int k = 0; k < 5; ++k) {
      *f[k] = (double *)p;
      p += up(bC);
    }
    slot[s].u = (double *)p;
    p += up(3 * bC) + up(bC);                    // u, and one spare field
    slot[s].R = p;
  }
  cudaStream_t cs = ctx->copy_stream, ks = ctx->stream, ms = ctx->mom_stream;
  auto h2d = [&](int i) {
    const rad_host_item &it = items[i];
    Slot &sl = slot[i & 1];
    cudaMemcpyAsync(sl.I, it.I, bI, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(sl.rho, it.rho, bC, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(sl.u, it.u, 3 * bC, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(sl.aa, it.alpha_a, bC, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(sl.as, it.alpha_s, bC, cudaMemcpyHostToDevice, cs);
    if (with_eta) cudaMemcpyAsync(sl.eta, it.eta, bC, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(sl.T, it.T, bC, cudaMemcpyHostToDevice, cs);
    cudaEventRecord(ctx->ev_h2d[i & 1], cs);
  };
  auto d2h = [&](int i) {
    const rad_host_item &it = items[i];
    Slot &sl = slot[i & 1];
    cudaStreamWaitEvent(cs, ctx->ev_done[i & 1], 0);
    cudaMemcpyAsync(it.R, sl.R, bR, cudaMemcpyDeviceToHost, cs);
    cudaMemcpyAsync(it.T, sl.T, bC, cudaMemcpyDeviceToHost, cs);
    if (it.I_out) cudaMemcpyAsync(it.I_out, sl.I, bI, cudaMemcpyDeviceToHost, cs);
  };
  // the copy and moment streams must not start before work already queued on
  // the context stream (an earlier call may still be using the slots)
  cudaEventRecord(ctx->ev_done[0], ks);
  cudaStreamWaitEvent(cs, ctx->ev_done[0], 0);
  cudaStreamWaitEvent(ms, ctx->ev_done[0], 0);
  h2d(0);
  int st = RAD_OK;
  for (int i = 0; i < n_items && st == RAD_OK; ++i) {
    if (i + 1 < n_items) {
      if (i >= 1) cudaStreamWaitEvent(cs, ctx->ev_done[(i + 1) & 1], 0);   // slot of item i - 1 released
      h2d(i + 1);
    }
    Slot &sl = slot[i & 1];
    cudaStreamWaitEvent(ks, ctx->ev_h2d[i & 1], 0);
    rad_gas g;
    g.rho = sl.rho;
    g.u = sl.u;
    g.alpha_a = sl.aa;
    g.alpha_s = sl.as;
    g.eta = with_eta ? sl.eta : nullptr;
    g.T = sl.T;
    for (int s = 0; s < nsteps && st == RAD_OK; ++s) st = rad_step(ctx, sl.I, &g, dt, o, nullptr);
    cudaEventRecord(ctx->ev_step[i & 1], ks);
    cudaStreamWaitEvent(ms, ctx->ev_step[i & 1], 0);
    if (st == RAD_OK) {
      std::string err;
      st = rad::launch_moments(ctx, sl.I, o->precision, frame, method, &g, sl.R, ms, err);
      if (st != RAD_OK) fail_h(ctx, st, err);
    }
    cudaEventRecord(ctx->ev_done[i & 1], ms);
    d2h(i);
  }
  cudaError_t ce = cudaStreamSynchronize(cs);
  cudaError_t me = cudaStreamSynchronize(ms);
  cudaError_t ke = cudaStreamSynchronize(ks);
  if (st != RAD_OK) return st;      // rad_step / the moments set the message
  if (ce != cudaSuccess || me != cudaSuccess || ke != cudaSuccess) {
    const cudaError_t e = ce != cudaSuccess ? ce : (me != cudaSuccess ? me : ke);
    return fail_h(ctx, RAD_ECUDA, std::string("rad_step_host: ") + cudaGetErrorString(e));
  }
  return RAD_OK;
}
