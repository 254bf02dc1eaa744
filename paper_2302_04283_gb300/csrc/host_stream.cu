// rad_step_host: the radiation step for data that lives in host memory.
//
// For each item the intensity and the gas state are copied to the device,
// advanced by rad_step, contracted by rad_moments, and the moments (plus the
// updated temperature and, on request, the intensity) are copied back.  Three
// device slots rotate, and four streams share the work: uploads (copy
// stream), steps (the context stream), moment contractions (moment stream)
// and read-backs (back stream).  Item i lives in slot i mod 3; its upload
// waits only until the item that held the slot before it (i - 3) has been
// contracted and read back, so the uploads of the next two items run while
// item i steps, and the read-backs use the other direction of the link
// concurrently.  With pinned host buffers the step rate is then set by the
// slower of the kernels and the upload.  The paper has no counterpart (it
// assumes the fields are resident).
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
  if (ctx->n_groups > 0) return fail_h(ctx, RAD_EUNSUPPORTED, "rad_step_host steps gray transport (no groups)");
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
  constexpr int NS = rad_ctx::kHostSlots;
  if (ctx->host_slot_bytes < NS * per_slot) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->host_slot_buf);
    ctx->host_slot_buf = nullptr;
    ctx->host_slot_bytes = 0;
    if (cudaMalloc(&ctx->host_slot_buf, NS * per_slot) != cudaSuccess)
      return fail_h(ctx, RAD_ENOMEM, "rad_step_host: slot allocation failed");
    ctx->host_slot_bytes = NS * per_slot;
  }
  if (!ctx->copy_stream) {
    if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->back_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->mom_stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail_h(ctx, RAD_ECUDA, "rad_step_host: stream creation failed");
    for (int s = 0; s < NS; ++s) {
      cudaEventCreateWithFlags(&ctx->ev_h2d[s], cudaEventDisableTiming);
      cudaEventCreateWithFlags(&ctx->ev_step[s], cudaEventDisableTiming);
      cudaEventCreateWithFlags(&ctx->ev_done[s], cudaEventDisableTiming);
      cudaEventCreateWithFlags(&ctx->ev_back[s], cudaEventDisableTiming);
    }
  }
  Slot slot[NS];
  for (int s = 0; s < NS; ++s) {
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
  cudaStream_t cs = ctx->copy_stream, bs = ctx->back_stream, ks = ctx->stream, ms = ctx->mom_stream;
  auto h2d = [&](int i) {
    const rad_host_item &it = items[i];
    const int s = i % NS;
    Slot &sl = slot[s];
    if (i >= NS) {   // item i - NS held the slot: its contraction and read-back must be over
      cudaStreamWaitEvent(cs, ctx->ev_done[s], 0);
      cudaStreamWaitEvent(cs, ctx->ev_back[s], 0);
    }
    cudaMemcpyAsync(sl.I, it.I, bI, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(sl.rho, it.rho, bC, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(sl.u, it.u, 3 * bC, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(sl.aa, it.alpha_a, bC, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(sl.as, it.alpha_s, bC, cudaMemcpyHostToDevice, cs);
    if (with_eta) cudaMemcpyAsync(sl.eta, it.eta, bC, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(sl.T, it.T, bC, cudaMemcpyHostToDevice, cs);
    cudaEventRecord(ctx->ev_h2d[s], cs);
  };
  auto d2h = [&](int i) {
    const rad_host_item &it = items[i];
    const int s = i % NS;
    Slot &sl = slot[s];
    cudaStreamWaitEvent(bs, ctx->ev_done[s], 0);
    cudaMemcpyAsync(it.R, sl.R, bR, cudaMemcpyDeviceToHost, bs);
    cudaMemcpyAsync(it.T, sl.T, bC, cudaMemcpyDeviceToHost, bs);
    if (it.I_out) cudaMemcpyAsync(it.I_out, sl.I, bI, cudaMemcpyDeviceToHost, bs);
    cudaEventRecord(ctx->ev_back[s], bs);
  };
  // the other streams must not start before work already queued on the
  // context stream (it may still be using device data the caller handed in)
  cudaEventRecord(ctx->ev_step[0], ks);
  cudaStreamWaitEvent(cs, ctx->ev_step[0], 0);
  cudaStreamWaitEvent(bs, ctx->ev_step[0], 0);
  cudaStreamWaitEvent(ms, ctx->ev_step[0], 0);
  for (int i = 0; i < NS - 1 && i < n_items; ++i) h2d(i);
  int st = RAD_OK;
  for (int i = 0; i < n_items && st == RAD_OK; ++i) {
    if (i + NS - 1 < n_items) h2d(i + NS - 1);
    const int s = i % NS;
    Slot &sl = slot[s];
    cudaStreamWaitEvent(ks, ctx->ev_h2d[s], 0);
    rad_gas g;
    g.rho = sl.rho;
    g.u = sl.u;
    g.alpha_a = sl.aa;
    g.alpha_s = sl.as;
    g.eta = with_eta ? sl.eta : nullptr;
    g.T = sl.T;
    for (int q = 0; q < nsteps && st == RAD_OK; ++q) st = rad_step(ctx, sl.I, &g, dt, o, nullptr);
    cudaEventRecord(ctx->ev_step[s], ks);
    cudaStreamWaitEvent(ms, ctx->ev_step[s], 0);
    if (st == RAD_OK) {
      std::string err;
      st = rad::launch_moments(ctx, sl.I, o->precision, frame, method, &g, sl.R, ms, err);
      if (st != RAD_OK) fail_h(ctx, st, err);
    }
    cudaEventRecord(ctx->ev_done[s], ms);
    d2h(i);
  }
  cudaError_t ce = cudaStreamSynchronize(cs);
  cudaError_t be = cudaStreamSynchronize(bs);
  cudaError_t me = cudaStreamSynchronize(ms);
  cudaError_t ke = cudaStreamSynchronize(ks);
  if (st != RAD_OK) return st;      // rad_step / the moments set the message
  if (ce != cudaSuccess || be != cudaSuccess || me != cudaSuccess || ke != cudaSuccess) {
    const cudaError_t e = ce != cudaSuccess ? ce : (be != cudaSuccess ? be : (me != cudaSuccess ? me : ke));
    return fail_h(ctx, RAD_ECUDA, std::string("rad_step_host: ") + cudaGetErrorString(e));
  }
  return RAD_OK;
}
