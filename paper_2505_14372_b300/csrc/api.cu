// C-ABI of libptycho: contexts, validation, scratch arena, launch sequences
// of the forward model, the adjoint and the gradient-descent step
// (arXiv 2505.14372 §3, §3.1, §3.2), grouping (§2.2) and kernel timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"
#include "errors.h"
#include "internal.h"
#include "ptycho.h"

using ptycho::EngineOps;
using ptycho::LaunchArgs;
using ptycho::ProblemDesc;

namespace {

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// most object blocks of the fused step end (k_step_tail)
constexpr int kTailMaxBlocks = 4096;

// Offsets of one call's scratch inside the context arena.
struct Layout {
  size_t Phat, A, w, gPhat, partials, stats, tail, stage_pos, stage_I, order, omax, wmax, waves, pA, pI, det, total;
};

Layout make_layout(const ptycho_geom& g, int B, bool store, int slots) {
  const size_t NP = (size_t)g.h * g.w;
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  L.Phat = take((size_t)g.K * NP * 8);
  L.A = take((size_t)B * g.K * NP * 8);
  L.w = take((size_t)B * NP * 4);
  L.gPhat = take((size_t)g.K * NP * 8);
  // loss partials: block sums of the loss kernel, or one per position for
  // the position-major kernel (two passes' worth for LSQML); then regulariser
  // and gradient-norm partials
  L.partials = take((size_t)(std::max(ptycho::kLossBlocks, 2 * B) + 3 * ptycho::kNormBlocks + 8) * 8);
  L.stats = take(4 * 8);
  // fused step end: its block counter and (at byte 128) the work queue of
  // the position-major launch, then one FP64 partial per block
  L.tail = take(256 + (size_t)(g.K + kTailMaxBlocks) * 8);
  L.stage_pos = take((size_t)B * 2 * 4);
  L.stage_I = take((size_t)B * NP * 4);
  L.order = take((size_t)B * 4);  // processing order of a position-major launch
  L.omax = take((size_t)g.S * 4);
  L.wmax = take((size_t)B * g.K * g.S * 4);
  const size_t esize = g.wave_prec ? 4 : 8;  // entry-wave copies: complex64 or two 16-bit parts
  // stored: every item's entry waves; recomputed: per cluster the entry waves
  // of all K modes of its position (plus one wave per mode for the LSQML
  // step pass), their far fields and the intensity
  L.waves = take(store ? (size_t)B * g.K * g.S * NP * esize : (size_t)slots * g.K * (g.S + 1) * NP * esize);
  L.pA = take(store ? 0 : (size_t)slots * g.K * NP * 8);
  L.pI = take(store ? 0 : (size_t)slots * NP * 4);
  // deterministic sums: every position's object patch gradient and probe
  // spectrum gradient, kept apart
  L.det = take(g.deterministic ? (size_t)B * (g.S + g.K) * NP * 8 : 0);
  L.total = off;
  return L;
}

}  // namespace

// Host checks of a geometry shared by every entry point that takes one
// (internal.h).
int ptycho::validate_geom(const ptycho_geom* g) {
  if (!g) return perr(PTYCHO_EINVAL, "geometry is NULL");
  if (g->S < 1 || g->K < 1) return perr(PTYCHO_EINVAL, "need S >= 1 and K >= 1");
  if (g->h != g->w) return perr(PTYCHO_EINVAL, "window must be square (h == w)");
  if (!ptycho::engine_for(g->h))
    return perr(PTYCHO_EINVAL, "window size " + std::to_string(g->h) + " not in {64, 128, 192, 256}");
  if (g->dft < 0 || g->dft > 4) return perr(PTYCHO_EINVAL, "unknown dft mode");
  if (g->dft != PTYCHO_DFT_FFT && !ptycho::engine_for(g->h, g->dft))
    return perr(PTYCHO_EINVAL, "the tensor-core DFT variants are built for the 192 x 192 window only");
  if (g->H < g->h || g->W < g->w) return perr(PTYCHO_EINVAL, "object smaller than the window");
  if (!(g->dx > 0) || !(g->lambda > 0) || !std::isfinite(g->dx) || !std::isfinite(g->lambda))
    return perr(PTYCHO_EINVAL, "dx and lambda must be finite and > 0");
  if (g->S > 1 && !g->dz) return perr(PTYCHO_EINVAL, "dz is NULL but S > 1");
  for (int i = 0; i + 1 < g->S; ++i)
    if (!std::isfinite(g->dz[i])) return perr(PTYCHO_EINVAL, "dz must be finite");
  if (!std::isfinite(g->bandlimit)) return perr(PTYCHO_EINVAL, "bandlimit must be finite");
  if (g->loss != PTYCHO_LOSS_AMPLITUDE && g->loss != PTYCHO_LOSS_POISSON && g->loss != PTYCHO_LOSS_GAUSSIAN)
    return perr(PTYCHO_EINVAL, "unknown loss");
  if (g->loss == PTYCHO_LOSS_GAUSSIAN && !(g->c > 0)) return perr(PTYCHO_EINVAL, "Gaussian loss needs sigma = c > 0");
  if (!(g->eps >= 0) || !(g->c >= 0)) return perr(PTYCHO_EINVAL, "eps and c must be >= 0");
  if (g->loss == PTYCHO_LOSS_POISSON && !(g->eps > 0)) return perr(PTYCHO_EINVAL, "Poisson loss needs eps > 0");
  if (g->loss == PTYCHO_LOSS_AMPLITUDE && !(g->eps + g->c > 0))
    return perr(PTYCHO_EINVAL, "amplitude loss needs eps + c > 0");
  if (g->waves < 0 || g->waves > 2) return perr(PTYCHO_EINVAL, "unknown waves mode");
  if (g->wave_prec < 0 || g->wave_prec > 2) return perr(PTYCHO_EINVAL, "unknown entry-wave storage format");
  if (g->wave_prec != PTYCHO_PREC_F32 && g->dft != PTYCHO_DFT_FFT)
    return perr(PTYCHO_EINVAL, "16-bit entry waves run with the FFT tile (dft = 0)");
  if (g->deterministic != 0 && g->deterministic != 1) return perr(PTYCHO_EINVAL, "deterministic must be 0 or 1");
  if (g->deterministic &&
      (g->waves == PTYCHO_WAVES_STORE || g->dft != PTYCHO_DFT_FFT || g->wave_prec != PTYCHO_PREC_F32))
    return perr(PTYCHO_EINVAL, "deterministic sums need recomputed waves, the FFT tile and FP32 entry waves");
  const double cells = (double)g->S * g->H * g->W;
  if (cells > 4.0e9) return perr(PTYCHO_EINVAL, "object too large");
  return PTYCHO_OK;
}

namespace {
using ptycho::validate_geom;

// Band-limit threshold on f_u^2 + f_v^2 (square window): the grid keeps
// (f_u w)^2 + (f_v h)^2 <= floor(x*x) with x = beta*h*w*0.5 in IEEE double.
int band_threshold(const ptycho_geom& g) {
  if (!(g.bandlimit > 0)) return -1;
  const double x = g.bandlimit * (double)g.h * (double)g.w * 0.5;
  const double T = std::floor(x * x);
  const double NN = (double)g.h * (double)g.h;
  const double q = std::floor(T / NN);
  return (int)std::min(q, 2.0e9);
}

}  // namespace

struct ptycho_ctx {
  ptycho_geom g{};
  std::vector<double> dz;
  const EngineOps* ops = nullptr;
  int N = 0, NP = 0, max_batch = 0, device = 0;
  float2* Hc = nullptr;
  int blT = -1;
  unsigned* status = nullptr;
  float2* gO = nullptr;
  float2* gP = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  bool store = true;
  int slots = 0;          // recompute slots (clusters of the recompute adjoint)
  int pos_clusters = 0;   // clusters of the position-major loss + adjoint (<= slots)
  char* lsq = nullptr;    // LSQML buffers, allocated on first use
  size_t lsq_bytes = 0;
  int res_fwd = 1, res_adj = 1, res_rec = 1;
  // host-buffer steps: the patterns after the first round of positions are
  // copied on their own stream while that round computes (split_B1 > 0
  // during such a step)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copied = nullptr;
  int split_B1 = 0;
  // Adam step count in device memory (ptycho_set_step_counter) and the bias
  // corrections of the current step
  int64_t* t_dev = nullptr;
  float* bc_dev = nullptr;
  // fused step end (single-CTA tiles): its grid, 0 when the tile has none.
  // A gradient step that ended with it leaves g_P^, g_O and the loss
  // partials cleared; call_seq counts the context's calls, and clean_after
  // names the call that may skip those memsets (the one right after such a
  // step, and never one that is being captured).
  int tail_grid = 0;
  unsigned long long call_seq = 0, clean_after = ~0ull;
  // timing
  int timing = 0;  // 0 off, 1 every kernel, 2 the tile kernels (forward / adjoint) only
  struct Pending {
    int kid;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  std::vector<std::string> names;
  std::vector<double> ms;
  std::vector<int> launches;
};

namespace {

int kernel_id(ptycho_ctx* c, const char* name) {
  for (size_t i = 0; i < c->names.size(); ++i)
    if (c->names[i] == name) return (int)i;
  c->names.emplace_back(name);
  c->ms.push_back(0.0);
  c->launches.push_back(0);
  return (int)c->names.size() - 1;
}

cudaEvent_t take_event(ptycho_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one launch with CUDA events on its stream when timing is on.
// Records a timing event on s; inside a stream capture as an external event
// node, so that every replay of the graph records its time.
void record_timing_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}

struct Timed {
  ptycho_ctx* c;
  cudaStream_t s;
  int kid = -1;
  cudaEvent_t a = nullptr;
  ptycho::Range range;
  Timed(ptycho_ctx* ctx, const char* name, cudaStream_t st) : c(ctx), s(st), range(name) {
    if (!c->timing) return;
    if (c->timing == 2 && std::strcmp(name, "adjoint") != 0 && std::strcmp(name, "forward") != 0) return;
    kid = kernel_id(c, name);
    a = take_event(c);
    record_timing_event(a, s);
  }
  ~Timed() {
    if (kid < 0) return;
    cudaEvent_t b = take_event(c);
    record_timing_event(b, s);
    c->pending.push_back({kid, a, b});
  }
};

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return perr(PTYCHO_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

ProblemDesc base_desc(ptycho_ctx* c, const Layout& L, const ptycho_c64* O, const float* pos, const int* idx,
                      int B, int npos) {
  ProblemDesc d{};
  d.O = reinterpret_cast<const float2*>(O);
  d.Phat = reinterpret_cast<const float2*>(c->arena + L.Phat);
  d.pos = pos;
  d.idx = idx;
  d.Hc = c->Hc;
  d.A = reinterpret_cast<float2*>(c->arena + L.A);
  d.w = reinterpret_cast<const float*>(c->arena + L.w);
  d.waves = c->store ? c->arena + L.waves : nullptr;
  d.gO = nullptr;
  d.gPhat = reinterpret_cast<float2*>(c->arena + L.gPhat);
  d.S = c->g.S;
  d.K = c->g.K;
  d.H = c->g.H;
  d.W = c->g.W;
  d.B = B;
  d.npos = npos;
  d.blT = c->blT;
  d.item0 = 0;
  return d;
}

LaunchArgs one_problem(ptycho_ctx* c, const Layout& L, const ProblemDesc& d) {
  LaunchArgs a{};
  a.d[0] = d;
  a.nd = 1;
  a.total = d.B * d.K;
  a.status = c->status;
  a.slots = c->arena + L.waves;
  a.slot_stride = (long long)c->g.S * c->NP * (c->g.wave_prec ? 4 : 8);
  return a;
}

// The position-major kernel counts positions, not items, and takes its slot
// as K entry-wave sets of S + 1 waves (the last for LSQML's probe direction).
LaunchArgs one_position_problem(ptycho_ctx* c, const Layout& L, const ProblemDesc& d) {
  LaunchArgs a = one_problem(c, L, d);
  a.total = d.B;
  a.slot_stride = (long long)c->g.K * (c->g.S + 1) * c->NP * (c->g.wave_prec ? 4 : 8);
  return a;
}
// A processing order pays only when the object does not sit in L2 anyway
// (then the clusters running at one time must share their patches there);
// below this size the extra launch would cost more than it saves.
constexpr size_t kOrderMinObjectBytes = 64ull << 20;
bool order_pays(size_t object_bytes) { return object_bytes > kOrderMinObjectBytes; }
size_t object_bytes(const ptycho_ctx* c) { return (size_t)c->g.S * c->g.H * c->g.W * 8; }

ptycho::PosArgs pos_args(ptycho_ctx* c, const Layout& L) {
  ptycho::PosArgs F{};
  F.Abuf = reinterpret_cast<float2*>(c->arena + L.pA);
  F.Ibuf = reinterpret_cast<float*>(c->arena + L.pI);
  F.astride = (long long)c->g.K * c->NP;
  F.queue = reinterpret_cast<unsigned*>(c->arena + L.tail + 128);
  return F;
}
void set_pos_loss(ProblemDesc& d, const float* Iexp, double* lpart, int model, const ptycho_geom& g) {
  d.Iexp = Iexp;
  d.lpart = lpart;
  d.model = model;
  d.eps = (float)g.eps;
  d.c = (float)g.c;
}

int check_call(ptycho_ctx* c, int B) {
  if (!c) return perr(PTYCHO_EINVAL, "context is NULL");
  ++c->call_seq;
  if (B < 0 || B > c->max_batch)
    return perr(PTYCHO_EINVAL, "B = " + std::to_string(B) + " outside [0, max_batch = " + std::to_string(c->max_batch) + "]");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) {
    cudaGetLastError();
    return perr(PTYCHO_EINVAL, "current CUDA device differs from the context's device");
  }
  return PTYCHO_OK;
}

// forward + loss + adjoint into (gO, gP); partials[0..nl) hold the loss.
// With gI != null the seed is the external cotangent dL/dI instead of the
// noise model's derivative (vector-Jacobian product).
// epie: the seed is the modulus update chi and the per-slice normalisers of
// §3.3.1 apply (gO, gP then hold the summed ePIE updates).
bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// fused_tail: the caller ends the step with k_step_tail, which computes the
// probe gradient itself (no probe_grad launch here); and if the previous
// call of this context was such a step (not under capture), g_P^, the
// context's g_O and the loss partials are already zero.
int run_gradient(ptycho_ctx* c, const ptycho_c64* O, const ptycho_c64* P, const float* pos, const int* idx, int B,
                 int npos, const float* Iexp, ptycho_c64* gO, ptycho_c64* gP, int accumulate, cudaStream_t s, int* nl_out,
                 bool vjp = false, const float* gI = nullptr, double* gpos = nullptr, bool epie = false,
                 bool fused_tail = false) {
  const Layout L = make_layout(c->g, c->max_batch, c->store, c->slots);
  const int K = c->g.K;
  float2* Phat = reinterpret_cast<float2*>(c->arena + L.Phat);
  float2* gPhat = reinterpret_cast<float2*>(c->arena + L.gPhat);
  double* partials = reinterpret_cast<double*>(c->arena + L.partials);
  const long long nO = (long long)c->g.S * c->g.H * c->g.W;
  {
    Timed t(c, "probe_spectrum", s);
    CK(c->ops->probe_spectrum(reinterpret_cast<const float2*>(P), Phat, K, s));
  }
  const bool clean = c->clean_after == c->call_seq && !capturing(s);
  if (!clean) CK(cudaMemsetAsync(gPhat, 0, (size_t)K * c->NP * 8, s));
  if (!accumulate && !(clean && reinterpret_cast<float2*>(gO) == c->gO)) CK(cudaMemsetAsync(gO, 0, (size_t)nO * 8, s));
  const int nl = (int)std::min<long long>(ptycho::kLossBlocks, std::max<long long>(1, ((long long)B * c->NP + 255) / 256));
  *nl_out = nl;
  if (B == 0) {
    CK(cudaMemsetAsync(partials, 0, (size_t)nl * 8, s));
    if (!accumulate) CK(cudaMemsetAsync(gP, 0, (size_t)K * c->NP * 8, s));
    return PTYCHO_OK;
  }
  ProblemDesc d = base_desc(c, L, O, pos, idx, B, npos);
  d.gO = reinterpret_cast<float2*>(gO);
  d.gpos = gpos;
  const int model = epie ? ptycho::kModelEpie : c->g.loss;
  if (epie) {
    unsigned* omax = reinterpret_cast<unsigned*>(c->arena + L.omax);
    d.omax = omax;
    d.wmax = reinterpret_cast<unsigned*>(c->arena + L.wmax);
    CK(cudaMemsetAsync(omax, 0, (size_t)c->g.S * 4, s));
    CK(cudaMemsetAsync(d.wmax, 0, (size_t)B * K * c->g.S * 4, s));
    Timed t(c, "slice_max", s);
    CK(ptycho::launch_slice_absmax(reinterpret_cast<const float2*>(O), c->g.S, (long long)c->g.H * c->g.W, omax, s));
  }
  // Entry waves recomputed: one position-major loss + adjoint launch (each
  // cluster takes whole scan positions, all modes in turn).  Deterministic
  // contexts keep every position's gradients apart and sum them afterwards
  // in position order.
  const bool det = c->g.deterministic && !epie && !vjp;
  const int variant = epie ? ptycho::kVarEpie : det ? ptycho::kVarDet : c->g.wave_prec;
  if (det) {
    d.det_gO = reinterpret_cast<float2*>(c->arena + L.det);
    d.det_gP = d.det_gO + (size_t)c->max_batch * c->g.S * c->NP;
  }
  if (gpos && !accumulate) CK(cudaMemsetAsync(gpos, 0, (size_t)B * 2 * sizeof(double), s));
  if (!c->store && !vjp && c->pos_clusters > 0) {
    ptycho::PosArgs F = pos_args(c, L);
    int* order = reinterpret_cast<int*>(c->arena + L.order);
    set_pos_loss(d, Iexp, partials, model, c->g);
    if (!clean) CK(cudaMemsetAsync(partials, 0, (size_t)B * 8, s));
    // split: positions [0, B1) first, then the rest once their patterns
    // (copied on another stream) are in; idx-free groups only
    const int B1 = (c->split_B1 > 0 && c->split_B1 < B && !idx && !det) ? c->split_B1 : B;
    {
      LaunchArgs la = one_position_problem(c, L, d);
      la.d[0].B = B1;
      la.total = B1;
      if (order_pays(object_bytes(c))) {
        CK(ptycho::launch_locality_order(la, order, s));
        F.order = order;
      }
      Timed t(c, "adjoint", s);
      CK(c->ops->adjoint_pos(la, F, std::min(B1, c->pos_clusters), variant, s));
    }
    if (B1 < B) {
      ProblemDesc d2 = d;
      d2.pos = pos + 2 * (size_t)B1;
      d2.Iexp = Iexp + (size_t)B1 * c->NP;
      d2.lpart = partials + B1;
      d2.B = B - B1;
      d2.npos = B - B1;
      LaunchArgs la2 = one_position_problem(c, L, d2);
      if (order_pays(object_bytes(c))) {
        CK(ptycho::launch_locality_order(la2, order + B1, s));
        F.order = order + B1;
      }
      CK(cudaStreamWaitEvent(s, c->copied, 0));
      Timed t(c, "adjoint", s);
      CK(c->ops->adjoint_pos(la2, F, std::min(B - B1, c->pos_clusters), variant, s));
    }
    *nl_out = B;
    if (det) {
      Timed t(c, "det_reduce", s);
      CK(ptycho::launch_det_reduce(d.det_gO, d.det_gP, pos, idx, npos, B, c->g.S, K, c->g.H, c->g.W, c->N,
                                   reinterpret_cast<float2*>(gO), gPhat, s));
    }
    if (fused_tail) return PTYCHO_OK;
    Timed t(c, "probe_grad", s);
    CK(c->ops->probe_grad(gPhat, reinterpret_cast<float2*>(gP), K, accumulate, s));
    return PTYCHO_OK;
  }
  LaunchArgs la = one_problem(c, L, d);
  const int items = B * K;
  if (order_pays(object_bytes(c))) {  // positions along a Hilbert curve, as in the position-major step
    int* order = reinterpret_cast<int*>(c->arena + L.order);
    CK(ptycho::launch_locality_order(one_position_problem(c, L, d), order, s));
    la.order = order;
  }
  {
    Timed t(c, "forward", s);
    CK(c->ops->forward(la, std::min(items, c->res_fwd), c->store, variant, s));
  }
  if (vjp) {
    Timed t(c, "seed", s);
    CK(c->ops->seed(gI, B, reinterpret_cast<float*>(c->arena + L.w), s));
  } else {
    Timed t(c, "loss", s);
    CK(c->ops->loss(d.A, Iexp, idx, npos, B, K, model, (float)c->g.eps, (float)c->g.c,
                    reinterpret_cast<float*>(c->arena + L.w), partials, nl, s));
  }
  {
    Timed t(c, "adjoint", s);
    // recomputing two-kernel path: one item per slot of S entry waves (the
    // region holds K of them per position slot)
    const int cl = c->store ? std::min(items, c->res_adj) : std::min({items, c->res_rec, c->slots * K});
    CK(c->ops->adjoint(la, cl, c->store, variant, s));
  }
  if (fused_tail) return PTYCHO_OK;
  {
    Timed t(c, "probe_grad", s);
    CK(c->ops->probe_grad(gPhat, reinterpret_cast<float2*>(gP), K, accumulate, s));
  }
  return PTYCHO_OK;
}

}  // namespace

// Context creation.  external_slots: the recompute scratch is supplied by
// the caller of every launch (the server shares one per window size), so the
// context holds none and always recomputes.
static int create_impl(const ptycho_geom* geom, int32_t max_batch, size_t scratch_budget_bytes, bool external_slots,
                       ptycho_ctx** out) {
  if (!out) return perr(PTYCHO_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate_geom(geom);
  if (rc) return rc;
  if (max_batch < 1) return perr(PTYCHO_EINVAL, "max_batch must be >= 1");
  if ((long long)max_batch * geom->K >= (1LL << 31)) return perr(PTYCHO_EINVAL, "max_batch * K too large");
  auto* c = new ptycho_ctx();
  c->g = *geom;
  c->dz.assign(geom->dz ? geom->dz : nullptr, geom->dz ? geom->dz + std::max(geom->S - 1, 0) : nullptr);
  c->g.dz = c->dz.data();
  c->ops = ptycho::engine_for(geom->h, geom->dft);
  c->N = geom->h;
  c->NP = geom->h * geom->w;
  c->max_batch = max_batch;
  c->blT = band_threshold(*geom);
  auto bail = [&](int code) {
    ptycho_destroy(c);
    return code;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return perr(PTYCHO_ECUDA, "no CUDA device");
  }
  const int var = geom->wave_prec;  // kVarF32 / kVarF16 / kVarBF16
  c->res_fwd = c->ops->resident_clusters(false, false, ptycho::kVarF32);
  c->res_rec = c->ops->resident_clusters(true, false, var);
  c->res_adj = c->ops->resident_clusters(true, true, var);
  // position slots: no more clusters than can run at once or than positions
  // in a call
  c->slots = std::max(1, std::min(c->res_rec, max_batch));
  c->pos_clusters = external_slots ? 0 : c->slots;
  // waves mode
  const Layout Ls = make_layout(c->g, max_batch, true, 0);
  const Layout Lr = make_layout(c->g, max_batch, false, external_slots ? 0 : c->slots);
  if (external_slots || geom->deterministic) c->store = false;
  else if (geom->waves == PTYCHO_WAVES_STORE) c->store = true;
  else if (geom->waves == PTYCHO_WAVES_RECOMPUTE) c->store = false;
  else c->store = scratch_budget_bytes == 0 || Ls.total <= scratch_budget_bytes;
  const Layout& L = c->store ? Ls : Lr;
  if (scratch_budget_bytes && L.total > scratch_budget_bytes)
    return bail(perr(PTYCHO_ENOMEM, "scratch needs " + std::to_string(L.total) + " bytes, budget is " +
                                        std::to_string(scratch_budget_bytes)));
  c->arena_bytes = L.total;
  if (cudaMalloc(&c->arena, c->arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    c->arena = nullptr;
    return bail(perr(PTYCHO_ENOMEM, "cudaMalloc of " + std::to_string(c->arena_bytes) + " scratch bytes failed"));
  }
  const size_t nO = (size_t)geom->S * geom->H * geom->W;
  if (cudaMalloc(&c->gO, nO * 8) != cudaSuccess || cudaMalloc(&c->gP, (size_t)geom->K * c->NP * 8) != cudaSuccess ||
      cudaMalloc(&c->status, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return bail(perr(PTYCHO_ENOMEM, "cudaMalloc of gradient buffers failed"));
  }
  if (cudaMemset(c->status, 0, sizeof(unsigned)) != cudaSuccess) return bail(perr(PTYCHO_ECUDA, "memset"));
  c->tail_grid = std::min(c->ops->tail_blocks((long long)nO, geom->K), geom->K + kTailMaxBlocks);
  if (cudaMemset(c->arena + L.tail, 0, 256) != cudaSuccess) return bail(perr(PTYCHO_ECUDA, "memset"));
  // separable Fresnel chirp per gap, in spectral slot order (FP64 phase in turns, reduced)
  if (geom->S > 1) {
    std::vector<float2> h((size_t)(geom->S - 1) * c->N);
    const int R1 = c->ops->R1, R2 = c->ops->R2, N = c->N;
    for (int s = 0; s + 1 < geom->S; ++s)
      for (int p = 0; p < N; ++p) {
        const int n = p / R2 + R1 * (p % R2);
        const double f = n < (N + 1) / 2 ? n : n - N;
        double t = geom->lambda * c->dz[s] * f * f / (2.0 * (double)N * N * geom->dx * geom->dx);
        t -= std::nearbyint(t);
        const double a = -2.0 * M_PI * t;
        h[(size_t)s * N + p] = make_float2((float)std::cos(a), (float)std::sin(a));
      }
    if (cudaMalloc(&c->Hc, h.size() * sizeof(float2)) != cudaSuccess ||
        cudaMemcpy(c->Hc, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return bail(perr(PTYCHO_ENOMEM, "propagator table allocation failed"));
    }
  }
  *out = c;
  return PTYCHO_OK;
}

extern "C" {

int ptycho_create(const ptycho_geom* geom, int32_t max_batch, size_t scratch_budget_bytes, ptycho_ctx** out) {
  return create_impl(geom, max_batch, scratch_budget_bytes, false, out);
}

int ptycho_destroy(ptycho_ctx* c) {
  if (!c) return PTYCHO_OK;
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  cudaFree(c->bc_dev);
  if (c->copied) cudaEventDestroy(c->copied);
  for (auto& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  cudaFree(c->arena);
  cudaFree(c->lsq);
  cudaFree(c->gO);
  cudaFree(c->gP);
  cudaFree(c->status);
  cudaFree(c->Hc);
  delete c;
  return PTYCHO_OK;
}

size_t ptycho_scratch_bytes(const ptycho_geom* geom, int32_t B, int32_t waves) {
  if (validate_geom(geom) || B < 0) return 0;
  const EngineOps* ops = ptycho::engine_for(geom->h);
  int slots = 148 / ops->G;
  int dev;
  if (cudaGetDevice(&dev) == cudaSuccess) slots = ops->resident_clusters(true, false, geom->wave_prec);
  else cudaGetLastError();
  slots = std::max(1, std::min(slots, B));
  return make_layout(*geom, B, waves != PTYCHO_WAVES_RECOMPUTE, slots).total;
}

int ptycho_forward(ptycho_ctx* c, const ptycho_c64* O, const ptycho_c64* P, const float* pos, int32_t B,
                   float* I_out, ptycho_stream stream) {
  ptycho::Range range("ptycho_forward");
  int rc = check_call(c, B);
  if (rc) return rc;
  if (B == 0) return PTYCHO_OK;
  if (!O || !P || !pos || !I_out) return perr(PTYCHO_EINVAL, "NULL array argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Layout L = make_layout(c->g, c->max_batch, c->store, c->slots);
  float2* Phat = reinterpret_cast<float2*>(c->arena + L.Phat);
  {
    Timed t(c, "probe_spectrum", s);
    CK(c->ops->probe_spectrum(reinterpret_cast<const float2*>(P), Phat, c->g.K, s));
  }
  ProblemDesc d = base_desc(c, L, O, pos, nullptr, B, B);
  d.waves = nullptr;
  LaunchArgs la = one_problem(c, L, d);
  if (order_pays(object_bytes(c))) {
    int* order = reinterpret_cast<int*>(c->arena + L.order);
    CK(ptycho::launch_locality_order(one_position_problem(c, L, d), order, s));
    la.order = order;
  }
  {
    Timed t(c, "forward", s);
    CK(c->ops->forward(la, std::min(B * c->g.K, c->res_fwd), false, ptycho::kVarF32, s));
  }
  {
    Timed t(c, "modesum", s);
    CK(c->ops->modesum(d.A, I_out, B, c->g.K, s));
  }
  return PTYCHO_OK;
}

int ptycho_adjoint(ptycho_ctx* c, const ptycho_c64* O, const ptycho_c64* P, const float* pos, int32_t B,
                   const float* I_exp, double* loss_out, ptycho_c64* gO, ptycho_c64* gP, int32_t accumulate,
                   ptycho_stream stream) {
  ptycho::Range range("ptycho_adjoint");
  int rc = check_call(c, B);
  if (rc) return rc;
  if (!O || !P || (B > 0 && (!pos || !I_exp)) || !gO || !gP) return perr(PTYCHO_EINVAL, "NULL array argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int nl = 0;
  rc = run_gradient(c, O, P, pos, nullptr, B, B, I_exp, gO, gP, accumulate, s, &nl);
  if (rc) return rc;
  if (loss_out) {
    const Layout L = make_layout(c->g, c->max_batch, c->store, c->slots);
    Timed t(c, "finalize", s);
    CK(ptycho::launch_finalize(reinterpret_cast<double*>(c->arena + L.partials), nl, 0, loss_out, 0, s));
  }
  return PTYCHO_OK;
}

int ptycho_adjoint_positions(ptycho_ctx* c, const ptycho_c64* O, const ptycho_c64* P, const float* pos, int32_t B,
                             const float* I_exp, double* loss_out, ptycho_c64* gO, ptycho_c64* gP, double* gpos_out,
                             int32_t accumulate, ptycho_stream stream) {
  ptycho::Range range("ptycho_adjoint_positions");
  int rc = check_call(c, B);
  if (rc) return rc;
  if (!O || !P || (B > 0 && (!pos || !I_exp || !gpos_out)) || !gO || !gP)
    return perr(PTYCHO_EINVAL, "NULL array argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int nl = 0;
  rc = run_gradient(c, O, P, pos, nullptr, B, B, I_exp, gO, gP, accumulate, s, &nl, false, nullptr, gpos_out);
  if (rc) return rc;
  if (loss_out) {
    const Layout L = make_layout(c->g, c->max_batch, c->store, c->slots);
    CK(ptycho::launch_finalize(reinterpret_cast<double*>(c->arena + L.partials), nl, 0, loss_out, 0, s));
  }
  return PTYCHO_OK;
}

int ptycho_vjp(ptycho_ctx* c, const ptycho_c64* O, const ptycho_c64* P, const float* pos, int32_t B,
               const float* gI, ptycho_c64* gO, ptycho_c64* gP, int32_t accumulate, ptycho_stream stream) {
  ptycho::Range range("ptycho_vjp");
  int rc = check_call(c, B);
  if (rc) return rc;
  if (!O || !P || (B > 0 && (!pos || !gI)) || !gO || !gP) return perr(PTYCHO_EINVAL, "NULL array argument");
  int nl = 0;
  return run_gradient(c, O, P, pos, nullptr, B, B, nullptr, gO, gP, accumulate, static_cast<cudaStream_t>(stream),
                      &nl, true, gI);
}

static int step_impl(ptycho_ctx* c, ptycho_c64* O, ptycho_c64* P, ptycho_adam* st, const ptycho_opt* opt,
                     const float* pos_all, const float* I_exp_all, int32_t n_pos, const int32_t* idx, int32_t B,
                     double* stats_out, cudaStream_t s) {
  if (!O || !P || !st || !opt || !st->mO || !st->vO || !st->mP || !st->vP)
    return perr(PTYCHO_EINVAL, "NULL argument");
  if (B > 0 && (!pos_all || !I_exp_all)) return perr(PTYCHO_EINVAL, "NULL positions or patterns");
  if (!(opt->beta1 >= 0 && opt->beta1 < 1 && opt->beta2 >= 0 && opt->beta2 < 1 && opt->eps >= 0 &&
        std::isfinite(opt->lr_O) && std::isfinite(opt->lr_P)))
    return perr(PTYCHO_EINVAL, "bad Adam parameters");
  const Layout L = make_layout(c->g, c->max_batch, c->store, c->slots);
  const bool tv0 = opt->reg_obj_tv != 0.f || opt->reg_obj_layers_tv != 0.f;
  const bool reg0 = opt->reg_obj_l2 != 0.f || opt->reg_obj_tikhonov != 0.f || opt->reg_obj_layers != 0.f ||
                    opt->reg_probe_l2 != 0.f || tv0;
  // single-CTA tiles without regularisers end the step in one fused launch
  const bool fused = c->tail_grid > 0 && !reg0;
  int nl = 0;
  int rc = run_gradient(c, O, P, pos_all, idx, B, n_pos, I_exp_all, reinterpret_cast<ptycho_c64*>(c->gO),
                        reinterpret_cast<ptycho_c64*>(c->gP), 0, s, &nl, false, nullptr, nullptr, false, fused);
  if (rc) return rc;
  double* partials = reinterpret_cast<double*>(c->arena + L.partials);
  double* stats = stats_out ? stats_out : reinterpret_cast<double*>(c->arena + L.stats);
  const long long nO = (long long)c->g.S * c->g.H * c->g.W;
  const long long nP = (long long)c->g.K * c->NP;
  const bool tv = opt->reg_obj_tv != 0.f || opt->reg_obj_layers_tv != 0.f;
  if (tv && !(opt->reg_tv_eps > 0.f)) return perr(PTYCHO_EINVAL, "TV regularisers need reg_tv_eps > 0");
  const bool reg = opt->reg_obj_l2 != 0.f || opt->reg_obj_tikhonov != 0.f || opt->reg_obj_layers != 0.f ||
                   opt->reg_probe_l2 != 0.f || tv;
  const int nr = reg ? ptycho::kNormBlocks : 0;
  if (reg) {
    Timed t(c, "regularize", s);
    CK(ptycho::launch_regularize(reinterpret_cast<const float2*>(O), c->gO, c->g.S, c->g.H, c->g.W,
                                 reinterpret_cast<const float2*>(P), c->gP, nP, opt->reg_obj_l2,
                                 opt->reg_obj_tikhonov, opt->reg_obj_layers, opt->reg_probe_l2, opt->reg_obj_tv,
                                 opt->reg_obj_layers_tv, opt->reg_tv_eps, partials + nl, nr, s));
  }
  const int64_t t = st->t + 1;
  const float bc1 = (float)(1.0 / (1.0 - std::pow((double)opt->beta1, (double)t)));
  const float bc2 = (float)(1.0 / (1.0 - std::pow((double)opt->beta2, (double)t)));
  if (fused) {
    Timed tm(c, "step_tail", s);
    const float* bcd = nullptr;
    if (c->t_dev) {
      CK(ptycho::launch_adam_count(reinterpret_cast<long long*>(c->t_dev), opt->beta1, opt->beta2, c->bc_dev, s));
      bcd = c->bc_dev;
    }
    ptycho::TailArgs A{};
    A.gPhat = reinterpret_cast<float2*>(c->arena + L.gPhat);
    A.P = reinterpret_cast<float2*>(P);
    A.mP = reinterpret_cast<float2*>(st->mP);
    A.vP = st->vP;
    A.O = reinterpret_cast<float2*>(O);
    A.mO = reinterpret_cast<float2*>(st->mO);
    A.vO = st->vO;
    A.gO = c->gO;
    A.nO = nO;
    A.K = c->g.K;
    A.update_probe = opt->update_probe ? 1 : 0;
    A.lrO = opt->lr_O;
    A.lrP = opt->lr_P;
    A.b1 = opt->beta1;
    A.b2 = opt->beta2;
    A.eps = opt->eps;
    A.bc1 = bc1;
    A.bc2 = bc2;
    A.bcd = bcd;
    A.lossp = partials;
    A.nl = nl;
    A.nz = std::max(nl, c->max_batch);
    A.normp = reinterpret_cast<double*>(c->arena + L.tail + 256);
    A.stats = stats;
    A.counter = reinterpret_cast<unsigned*>(c->arena + L.tail);
    CK(c->ops->step_tail(A, c->tail_grid, s));
    if (!capturing(s)) c->clean_after = c->call_seq + 1;
    st->t = t;
    return PTYCHO_OK;
  }
  {
    // the Adam launches also write the |g|^2 partials of the gradients they read
    Timed tm(c, "adam", s);
    const float* bcd = nullptr;
    if (c->t_dev) {
      CK(ptycho::launch_adam_count(reinterpret_cast<long long*>(c->t_dev), opt->beta1, opt->beta2, c->bc_dev, s));
      bcd = c->bc_dev;
    }
    double* normO = partials + nl + nr;
    double* normP = normO + ptycho::kNormBlocks;
    CK(ptycho::launch_adam(reinterpret_cast<float2*>(O), reinterpret_cast<float2*>(st->mO), st->vO, c->gO, nO,
                           opt->lr_O, opt->beta1, opt->beta2, opt->eps, bc1, bc2, s, bcd, normO));
    if (opt->update_probe)
      CK(ptycho::launch_adam(reinterpret_cast<float2*>(P), reinterpret_cast<float2*>(st->mP), st->vP, c->gP, nP,
                             opt->lr_P, opt->beta1, opt->beta2, opt->eps, bc1, bc2, s, bcd, normP));
    else
      CK(ptycho::launch_sumsq(c->gP, nP, normP, ptycho::kNormBlocks, s));
    CK(ptycho::launch_finalize(partials, nl + nr, 2 * ptycho::kNormBlocks, stats, 1, s));
  }
  st->t = t;
  return PTYCHO_OK;
}

int ptycho_step(ptycho_ctx* c, ptycho_c64* O, ptycho_c64* P, ptycho_adam* st, const ptycho_opt* opt,
                const float* pos_all, const float* I_exp_all, int32_t n_pos, const int32_t* idx, int32_t B,
                double* stats_out, ptycho_stream stream) {
  ptycho::Range range("ptycho_step");
  int rc = check_call(c, B);
  if (rc) return rc;
  if (B > 0 && !idx) return perr(PTYCHO_EINVAL, "idx is NULL");
  if (n_pos < 0) return perr(PTYCHO_EINVAL, "n_pos < 0");
  return step_impl(c, O, P, st, opt, pos_all, I_exp_all, n_pos, idx, B, stats_out, static_cast<cudaStream_t>(stream));
}

int ptycho_step_host(ptycho_ctx* c, ptycho_c64* O, ptycho_c64* P, ptycho_adam* st, const ptycho_opt* opt,
                     const float* pos_host, const float* I_exp_host, int32_t B, double* loss_host,
                     double* gnorm_host, ptycho_stream stream) {
  ptycho::Range range("ptycho_step_host");
  int rc = check_call(c, B);
  if (rc) return rc;
  if (B > 0 && (!pos_host || !I_exp_host)) return perr(PTYCHO_EINVAL, "NULL host arrays");
  for (int j = 0; j < B; ++j) {
    const double y = std::floor((double)pos_host[2 * j] + 0.5), x = std::floor((double)pos_host[2 * j + 1] + 0.5);
    if (!(y >= 0 && x >= 0 && y + c->N <= c->g.H && x + c->N <= c->g.W))
      return perr(PTYCHO_EOUTOFBOUNDS, "scan position " + std::to_string(j) + " leaves the object");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Layout L = make_layout(c->g, c->max_batch, c->store, c->slots);
  float* dpos = reinterpret_cast<float*>(c->arena + L.stage_pos);
  float* dI = reinterpret_cast<float*>(c->arena + L.stage_I);
  double* stats = reinterpret_cast<double*>(c->arena + L.stats);
  // With the position-major step and more than one round of positions, only
  // the first round's patterns are copied ahead of the compute; the rest
  // travel on the context's copy stream while that round runs.
  int B1 = B;
  if (!c->store && c->pos_clusters > 0 && B > c->pos_clusters && !c->g.deterministic) {
    if (!c->copy_stream) {
      CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&c->copied, cudaEventDisableTiming));
    }
    B1 = c->pos_clusters;
  }
  if (B > 0) {
    Timed t(c, "h2d", s);
    CK(cudaMemcpyAsync(dpos, pos_host, (size_t)B * 2 * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dI, I_exp_host, (size_t)B1 * c->NP * 4, cudaMemcpyHostToDevice, s));
  }
  if (B1 < B) {
    // the staging rows are free: the previous call synchronised its stream
    CK(cudaMemcpyAsync(dI + (size_t)B1 * c->NP, I_exp_host + (size_t)B1 * c->NP, (size_t)(B - B1) * c->NP * 4,
                       cudaMemcpyHostToDevice, c->copy_stream));
    CK(cudaEventRecord(c->copied, c->copy_stream));
    c->split_B1 = B1;
  }
  rc = step_impl(c, O, P, st, opt, dpos, dI, B, nullptr, B, stats, s);
  c->split_B1 = 0;
  if (rc) {
    if (B1 < B) cudaStreamSynchronize(c->copy_stream);
    return rc;
  }
  double h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, stats, 16, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (loss_host) *loss_host = h[0];
  if (gnorm_host) *gnorm_host = h[1];
  return PTYCHO_OK;
}

int ptycho_epie_step(ptycho_ctx* c, ptycho_c64* O, ptycho_c64* P, float beta_O, float beta_P, const float* pos_all,
                     const float* I_exp_all, int32_t n_pos, const int32_t* idx, int32_t B, double* loss_out,
                     ptycho_stream stream) {
  ptycho::Range range("ptycho_epie_step");
  int rc = check_call(c, B);
  if (rc) return rc;
  if (!O || !P) return perr(PTYCHO_EINVAL, "NULL object or probe");
  if (B > 0 && (!idx || !pos_all || !I_exp_all)) return perr(PTYCHO_EINVAL, "NULL positions, patterns or idx");
  if (n_pos < 0) return perr(PTYCHO_EINVAL, "n_pos < 0");
  if (c->g.loss != PTYCHO_LOSS_AMPLITUDE)
    return perr(PTYCHO_EINVAL, "ePIE needs the amplitude / Anscombe noise model");
  if (!c->ops->has_variants || c->g.wave_prec != PTYCHO_PREC_F32)
    return perr(PTYCHO_EINVAL, "ePIE runs with the FFT tile (dft = 0) and FP32 entry waves");
  if (!std::isfinite(beta_O) || !std::isfinite(beta_P)) return perr(PTYCHO_EINVAL, "step sizes must be finite");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Layout L = make_layout(c->g, c->max_batch, c->store, c->slots);
  int nl = 0;
  rc = run_gradient(c, O, P, pos_all, idx, B, n_pos, I_exp_all, reinterpret_cast<ptycho_c64*>(c->gO),
                    reinterpret_cast<ptycho_c64*>(c->gP), 0, s, &nl, false, nullptr, nullptr, true);
  if (rc) return rc;
  if (loss_out) {
    Timed t(c, "finalize", s);
    CK(ptycho::launch_finalize(reinterpret_cast<double*>(c->arena + L.partials), nl, 0, loss_out, 0, s));
  }
  if (B == 0) return PTYCHO_OK;
  Timed t(c, "epie_apply", s);
  CK(ptycho::launch_axpy(reinterpret_cast<float2*>(O), c->gO, (long long)c->g.S * c->g.H * c->g.W, beta_O, s));
  if (beta_P != 0.f)
    CK(ptycho::launch_axpy(reinterpret_cast<float2*>(P), c->gP, (long long)c->g.K * c->NP, beta_P / (float)B, s));
  return PTYCHO_OK;
}

int ptycho_lsqml_step(ptycho_ctx* c, ptycho_c64* O, ptycho_c64* P, const ptycho_lsqml_opt* opt,
                      const float* illum_prev, const float* trans_prev, float* illum_acc, float* trans_acc,
                      const float* pos_all, const float* I_exp_all, int32_t n_pos, const int32_t* idx, int32_t B,
                      double* loss_out, ptycho_stream stream) {
  ptycho::Range range("ptycho_lsqml_step");
  int rc = check_call(c, B);
  if (rc) return rc;
  if (!O || !P || !opt) return perr(PTYCHO_EINVAL, "NULL object, probe or options");
  if (B > 0 && (!idx || !pos_all || !I_exp_all)) return perr(PTYCHO_EINVAL, "NULL positions, patterns or idx");
  if (n_pos < 0) return perr(PTYCHO_EINVAL, "n_pos < 0");
  if (c->g.loss != PTYCHO_LOSS_AMPLITUDE)
    return perr(PTYCHO_EINVAL, "LSQML needs the amplitude / Anscombe noise model");
  if (c->store || c->pos_clusters <= 0 || !c->ops->has_variants || c->g.wave_prec != PTYCHO_PREC_F32)
    return perr(PTYCHO_EINVAL, "LSQML runs with recomputed FP32 entry waves and the FFT tile");
  if (!(std::isfinite(opt->beta_O) && std::isfinite(opt->beta_P) && opt->delta_O >= 0.f && opt->delta_P >= 0.f &&
        opt->gamma >= 0.f))
    return perr(PTYCHO_EINVAL, "bad LSQML options");
  if (B == 0) return PTYCHO_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int K = c->g.K, S = c->g.S;
  const long long NP = c->NP, nO = (long long)S * c->g.H * c->g.W;
  // buffers: illumination, step-weighted illumination, object direction,
  // transmission (plain, weighted), probe direction and its spectra, sums
  const size_t sz_il = align256((size_t)nO * 4), sz_dO = align256((size_t)nO * 8), sz_T = align256((size_t)NP * 4),
               sz_dP = align256((size_t)K * NP * 8), sz_sum = align256((size_t)c->max_batch * S * 8),
               sz_sumP = align256((size_t)c->max_batch * 8);
  const size_t need = 2 * sz_il + sz_dO + 2 * sz_T + 2 * sz_dP + 2 * sz_sum + 2 * sz_sumP;
  if (!c->lsq) {
    if (cudaMalloc(&c->lsq, need) != cudaSuccess) {
      cudaGetLastError();
      c->lsq = nullptr;
      return perr(PTYCHO_ENOMEM, "cudaMalloc of " + std::to_string(need) + " LSQML bytes failed");
    }
    c->lsq_bytes = need;
  }
  char* q = c->lsq;
  float* il = reinterpret_cast<float*>(q);
  float* aw = reinterpret_cast<float*>(q += sz_il);
  float2* dO = reinterpret_cast<float2*>(q += sz_il);
  float* T = reinterpret_cast<float*>(q += sz_dO);
  float* AT = reinterpret_cast<float*>(q += sz_T);
  float2* dP = reinterpret_cast<float2*>(q += sz_T);
  float2* dPhat = reinterpret_cast<float2*>(q += sz_dP);
  double* num = reinterpret_cast<double*>(q += sz_dP);
  double* den = reinterpret_cast<double*>(q += sz_sum);
  double* numP = reinterpret_cast<double*>(q += sz_sum);
  double* denP = reinterpret_cast<double*>(q += sz_sumP);

  const Layout L = make_layout(c->g, c->max_batch, c->store, c->slots);
  float2* Phat = reinterpret_cast<float2*>(c->arena + L.Phat);
  float2* gPhat = reinterpret_cast<float2*>(c->arena + L.gPhat);
  double* partials = reinterpret_cast<double*>(c->arena + L.partials);
  ptycho::PosArgs F = pos_args(c, L);
  F.gamma = opt->gamma;
  const int clusters = std::min((int)B, c->pos_clusters);

  // pass 1: update directions (into gO, gP) and the group's illumination
  {
    Timed t(c, "probe_spectrum", s);
    CK(c->ops->probe_spectrum(reinterpret_cast<const float2*>(P), Phat, K, s));
  }
  CK(cudaMemsetAsync(gPhat, 0, (size_t)K * NP * 8, s));
  CK(cudaMemsetAsync(c->gO, 0, (size_t)nO * 8, s));
  CK(cudaMemsetAsync(il, 0, (size_t)nO * 4, s));
  CK(cudaMemsetAsync(T, 0, (size_t)NP * 4, s));
  CK(cudaMemsetAsync(partials, 0, (size_t)B * 8, s));
  ProblemDesc d = base_desc(c, L, O, pos_all, idx, B, n_pos);
  d.gO = c->gO;
  d.lsq_il = il;
  set_pos_loss(d, I_exp_all, partials, ptycho::kModelEpie, c->g);  // the modulus-update seed
  LaunchArgs la = one_position_problem(c, L, d);
  // both passes take the group's positions in the same locality order
  if (order_pays(object_bytes(c))) {
    CK(ptycho::launch_locality_order(la, reinterpret_cast<int*>(c->arena + L.order), s));
    F.order = reinterpret_cast<const int*>(c->arena + L.order);
  }
  {
    Timed t(c, "adjoint", s);
    CK(c->ops->adjoint_pos(la, F, clusters, ptycho::kVarLsqDir, s));
  }
  {
    Timed t(c, "probe_grad", s);
    CK(c->ops->probe_grad(gPhat, c->gP, K, 0, s));
  }
  if (loss_out) CK(ptycho::launch_finalize(partials, B, 0, loss_out, 0, s));
  {
    Timed t(c, "lsq_host_terms", s);
    CK(ptycho::launch_transmission(reinterpret_cast<const float2*>(O), S, c->g.H, c->g.W, c->N, pos_all, idx, n_pos, B,
                                   nullptr, nullptr, 0.f, T, s));
    if (illum_acc) CK(ptycho::launch_add(illum_acc, il, nO, s));
    if (trans_acc) CK(ptycho::launch_add(trans_acc, T, NP, s));
    CK(ptycho::launch_divide(c->gO, il, illum_prev, opt->delta_O, nO, nO, dO, s));
    CK(ptycho::launch_divide(c->gP, T, trans_prev, opt->delta_P, (long long)K * NP, NP, dP, s));
  }
  {
    Timed t(c, "probe_spectrum", s);
    CK(c->ops->probe_spectrum(dP, dPhat, K, s));
  }
  // pass 2: per-position step sizes and the step-weighted illumination
  CK(cudaMemsetAsync(num, 0, (size_t)B * S * 8, s));
  CK(cudaMemsetAsync(den, 0, (size_t)B * S * 8, s));
  CK(cudaMemsetAsync(numP, 0, (size_t)B * 8, s));
  CK(cudaMemsetAsync(denP, 0, (size_t)B * 8, s));
  CK(cudaMemsetAsync(aw, 0, (size_t)nO * 4, s));
  CK(cudaMemsetAsync(AT, 0, (size_t)NP * 4, s));
  ProblemDesc d2 = base_desc(c, L, O, pos_all, idx, B, n_pos);
  set_pos_loss(d2, I_exp_all, partials + B, ptycho::kModelEpie, c->g);  // the loss of this pass is not used
  d2.gO = c->gO;
  d2.lsq_dO = dO;
  d2.lsq_dPhat = dPhat;
  d2.lsq_num = num;
  d2.lsq_den = den;
  d2.lsq_numP = numP;
  d2.lsq_denP = denP;
  d2.lsq_aw = aw;
  LaunchArgs la2 = one_position_problem(c, L, d2);
  CK(cudaMemsetAsync(d2.lpart, 0, (size_t)B * 8, s));
  {
    Timed t(c, "adjoint", s);
    CK(c->ops->adjoint_pos(la2, F, clusters, ptycho::kVarLsqStep, s));
  }
  {
    Timed t(c, "lsq_update", s);
    CK(ptycho::launch_transmission(reinterpret_cast<const float2*>(O), S, c->g.H, c->g.W, c->N, pos_all, idx, n_pos, B,
                                   numP, denP, opt->gamma, AT, s));
    CK(ptycho::launch_weighted_update(reinterpret_cast<float2*>(O), dO, aw, il, opt->beta_O, nO, nO, s));
    CK(ptycho::launch_weighted_update(reinterpret_cast<float2*>(P), dP, AT, T, opt->beta_P, (long long)K * NP, NP, s));
  }
  return PTYCHO_OK;
}

int ptycho_check(ptycho_ctx* c, ptycho_stream stream) {
  if (!c) return perr(PTYCHO_EINVAL, "context is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaStreamSynchronize(s));
  unsigned st = 0;
  CK(cudaMemcpy(&st, c->status, sizeof(st), cudaMemcpyDeviceToHost));
  CK(cudaMemset(c->status, 0, sizeof(unsigned)));
  if (const unsigned bits = c->ops->take_check_bits())
    return perr(PTYCHO_ECHECK, "checked build: an index check failed (bits " + std::to_string(bits) +
                                   ": 1 shared-memory slot, 2 window coordinate, 4 item); the access was skipped");
  if (c->ops->take_exchange_timeouts())
    return perr(PTYCHO_ETIMEDOUT, "a bounded wait of the cluster exchange ran out; the last results are not valid");
  if (st & ptycho::PTYCHO_STATUS_OUT_OF_BOUNDS)
    return perr(PTYCHO_EOUTOFBOUNDS, "a scan window left the object; its item was skipped");
  return PTYCHO_OK;
}

int ptycho_set_timing(ptycho_ctx* c, int32_t enable) {
  if (!c) return perr(PTYCHO_EINVAL, "context is NULL");
  if (enable < 0 || enable > 2) return perr(PTYCHO_EINVAL, "timing mode must be 0, 1 or 2");
  c->timing = enable;
  return PTYCHO_OK;
}

int ptycho_kernel_times(ptycho_ctx* c, const char** names, double* ms, int32_t* launches, int32_t cap) {
  if (!c) return perr(PTYCHO_EINVAL, "context is NULL");
  for (auto& p : c->pending) {
    float f = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&f, p.a, p.b) == cudaSuccess) {
      c->ms[p.kid] += f;
      c->launches[p.kid] += 1;
    } else {
      cudaGetLastError();
    }
    c->pool.push_back(p.a);
    c->pool.push_back(p.b);
  }
  c->pending.clear();
  const int n = (int)c->names.size();
  if (cap < 0) {  // reset
    std::fill(c->ms.begin(), c->ms.end(), 0.0);
    std::fill(c->launches.begin(), c->launches.end(), 0);
    return n;
  }
  for (int i = 0; i < std::min(n, (int)cap); ++i) {
    if (names) names[i] = c->names[i].c_str();
    if (ms) ms[i] = c->ms[i];
    if (launches) launches[i] = c->launches[i];
  }
  return n;
}

int ptycho_fft2(int32_t N, int32_t dir, const ptycho_c64* in, ptycho_c64* out, int32_t count, ptycho_stream stream) {
  ptycho::Range range("ptycho_fft2");
  const EngineOps* ops = ptycho::engine_for(N);
  if (!ops) return perr(PTYCHO_EINVAL, "N not in {64, 128, 192, 256}");
  if (dir == 0 || count < 0 || (count > 0 && (!in || !out))) return perr(PTYCHO_EINVAL, "bad arguments");
  if (count == 0) return PTYCHO_OK;
  CK(ops->fft_debug(reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out), count, dir,
                    static_cast<cudaStream_t>(stream)));
  return PTYCHO_OK;
}

int ptycho_fft2_dft(int32_t N, int32_t dft, int32_t dir, const ptycho_c64* in, ptycho_c64* out, int32_t count,
                    ptycho_stream stream) {
  ptycho::Range range("ptycho_fft2_dft");
  if (dft < 0 || dft > 4) return perr(PTYCHO_EINVAL, "unknown dft mode");
  const EngineOps* ops = ptycho::engine_for(N, dft);
  if (!ops) return perr(PTYCHO_EINVAL, "no tile for this N and dft mode");
  if (dir == 0 || count < 0 || (count > 0 && (!in || !out))) return perr(PTYCHO_EINVAL, "bad arguments");
  if (count == 0) return PTYCHO_OK;
  CK(ops->fft_debug(reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out), count, dir,
                    static_cast<cudaStream_t>(stream)));
  return PTYCHO_OK;
}

int ptycho_exchange_selftest(int32_t N) {
  const EngineOps* ops = ptycho::engine_for(N);
  if (!ops) return perr(PTYCHO_EINVAL, "N not in {64, 128, 192, 256}");
  if (ops->G != 2) return perr(PTYCHO_EINVAL, "only the 192 x 192 tile exchanges through mbarriers");
  ops->take_exchange_timeouts();  // clear
  CK(ops->exchange_probe(nullptr));
  CK(cudaDeviceSynchronize());
  if (ops->take_exchange_timeouts())
    return perr(PTYCHO_ETIMEDOUT, "the exchange wait gave up as the self-test expects");
  return PTYCHO_OK;
}

int ptycho_set_step_counter(ptycho_ctx* c, int64_t* t_dev) {
  int rc = check_call(c, 0);
  if (rc) return rc;
  if (t_dev && !c->bc_dev) {
    if (cudaMalloc(&c->bc_dev, 2 * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      c->bc_dev = nullptr;
      return perr(PTYCHO_ENOMEM, "no device memory for the bias corrections");
    }
  }
  c->t_dev = t_dev;
  return PTYCHO_OK;
}

const char* ptycho_version(void) { return "libptycho 0.1 (sm_103a)"; }
int32_t ptycho_build_checked(void) { return PTYCHO_CHECKED ? 1 : 0; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Internal API for the serving runtime (internal.h).
namespace ptycho {

int ctx_create_shared_slots(const ptycho_geom* geom, int max_batch, ptycho_ctx** out) {
  return create_impl(geom, max_batch, 0, true, out);
}

size_t ctx_device_bytes(const ptycho_ctx* c) {
  const size_t nO = (size_t)c->g.S * c->g.H * c->g.W;
  return c->arena_bytes + nO * 8 + (size_t)c->g.K * c->NP * 8 + (c->g.S > 1 ? (size_t)(c->g.S - 1) * c->N * 8 : 0);
}

int resident_slots(int N) {
  const EngineOps* ops = engine_for(N);
  return ops ? ops->resident_clusters(true, false, kVarF32) : 0;
}

// positions of one served launch that get a processing order
constexpr int kOrderCap = kMaxDesc * 4096;
size_t pos_scratch_bytes(int N, int kmodes, int smax) {
  const size_t NP = (size_t)N * N, cl = (size_t)resident_slots(N);
  return cl * ((size_t)kmodes * (smax + 1) * NP * 8 + (size_t)kmodes * NP * 8 + NP * 4) + (size_t)kOrderCap * 4 + 256;
}
PosScratch pos_scratch_at(char* base, int N, int kmodes, int smax) {
  PosScratch p;
  const size_t NP = (size_t)N * N;
  p.clusters = resident_slots(N);
  p.kmodes = kmodes;
  p.smax = smax;
  p.slot_bytes = (long long)kmodes * (smax + 1) * NP * 8;
  p.slots = base;
  p.A = reinterpret_cast<float2*>(base + (size_t)p.clusters * p.slot_bytes);
  p.I = reinterpret_cast<float*>(reinterpret_cast<char*>(p.A) + (size_t)p.clusters * kmodes * NP * 8);
  p.order = reinterpret_cast<int*>(p.I + (size_t)p.clusters * NP);
  p.order_cap = kOrderCap;
  p.queue = reinterpret_cast<unsigned*>(p.order + kOrderCap);
  return p;
}

namespace {

// Adam, norms and regularisers of one job after its gradient launch(es);
// nl: loss partials at the start of its partials.
int finish_job(const StepJob& J, const Layout& L, int nl, cudaStream_t s) {
  ptycho_ctx* c = J.c;
  double* partials = reinterpret_cast<double*>(c->arena + L.partials);
  const long long nO = (long long)c->g.S * c->g.H * c->g.W, nP = (long long)c->g.K * c->NP;
  CK(c->ops->probe_grad(reinterpret_cast<float2*>(c->arena + L.gPhat), c->gP, c->g.K, 0, s));
  const bool reg = J.opt.reg_obj_l2 != 0.f || J.opt.reg_obj_tikhonov != 0.f || J.opt.reg_obj_layers != 0.f ||
                   J.opt.reg_probe_l2 != 0.f || J.opt.reg_obj_tv != 0.f || J.opt.reg_obj_layers_tv != 0.f;
  const int nr = reg ? kNormBlocks : 0;
  if (reg)
    CK(launch_regularize(J.O, c->gO, c->g.S, c->g.H, c->g.W, J.P, c->gP, nP, J.opt.reg_obj_l2, J.opt.reg_obj_tikhonov,
                         J.opt.reg_obj_layers, J.opt.reg_probe_l2, J.opt.reg_obj_tv, J.opt.reg_obj_layers_tv,
                         J.opt.reg_tv_eps, partials + nl, nr, s));
  const double t = (double)J.t;
  const float bc1 = (float)(1.0 / (1.0 - std::pow((double)J.opt.beta1, t)));
  const float bc2 = (float)(1.0 / (1.0 - std::pow((double)J.opt.beta2, t)));
  // the Adam launches also write the |g|^2 partials of the gradients they read
  double* normO = partials + nl + nr;
  double* normP = normO + kNormBlocks;
  CK(launch_adam(J.O, J.mO, J.vO, c->gO, nO, J.opt.lr_O, J.opt.beta1, J.opt.beta2, J.opt.eps, bc1, bc2, s, nullptr,
                 normO));
  if (J.opt.update_probe)
    CK(launch_adam(J.P, J.mP, J.vP, c->gP, nP, J.opt.lr_P, J.opt.beta1, J.opt.beta2, J.opt.eps, bc1, bc2, s, nullptr,
                   normP));
  else
    CK(launch_sumsq(c->gP, nP, normP, kNormBlocks, s));
  CK(launch_finalize(partials, nl + nr, 2 * kNormBlocks, J.stats, 1, s));
  return PTYCHO_OK;
}

// All jobs in one position-major loss + adjoint launch.
int step_batch_pos(const StepJob* jobs, int n, const PosScratch& ps, unsigned* status, cudaStream_t s) {
  const EngineOps* ops = jobs[0].c->ops;
  LaunchArgs la{};
  la.nd = n;
  la.status = status;
  la.slots = ps.slots;
  la.slot_stride = ps.slot_bytes;
  std::vector<Layout> L(n);
  // the costliest positions (most slices times modes) first in the launch's
  // order: the clusters claim positions in that order, so the cheap ones
  // fill in at the end
  std::vector<int> by_cost(n);
  for (int i = 0; i < n; ++i) by_cost[i] = i;
  auto cost = [&](int i) { return (long long)jobs[i].c->g.K * (2LL * jobs[i].c->g.S + 1); };
  std::stable_sort(by_cost.begin(), by_cost.end(), [&](int a, int b) { return cost(a) > cost(b); });
  int total = 0;
  for (int q = 0; q < n; ++q) {
    const int i = by_cost[q];
    const StepJob& J = jobs[i];
    ptycho_ctx* c = J.c;
    L[i] = make_layout(c->g, c->max_batch, false, 0);
    CK(ops->probe_spectrum(J.P, reinterpret_cast<float2*>(c->arena + L[i].Phat), c->g.K, s));
    CK(cudaMemsetAsync(c->arena + L[i].gPhat, 0, (size_t)c->g.K * c->NP * 8, s));
    CK(cudaMemsetAsync(c->gO, 0, (size_t)c->g.S * c->g.H * c->g.W * 8, s));
    double* partials = reinterpret_cast<double*>(c->arena + L[i].partials);
    CK(cudaMemsetAsync(partials, 0, (size_t)J.B * 8, s));
    ProblemDesc d = base_desc(c, L[i], reinterpret_cast<const ptycho_c64*>(J.O), J.pos, J.idx, J.B, J.n_pos);
    d.gO = c->gO;
    d.item0 = total;
    set_pos_loss(d, J.Iexp, partials, c->g.loss, c->g);
    total += J.B;
    la.d[q] = d;
  }
  la.total = total;
  PosArgs F{};
  F.queue = ps.queue;
  F.Abuf = ps.A;
  F.Ibuf = ps.I;
  F.astride = (long long)ps.kmodes * jobs[0].c->NP;
  size_t objects = 0;
  for (int i = 0; i < n; ++i) objects += object_bytes(jobs[i].c);
  if (ps.order && total <= ps.order_cap && order_pays(objects)) {  // each job's positions along a Hilbert curve
    CK(launch_locality_order(la, ps.order, s));
    F.order = ps.order;
  }
  CK(ops->adjoint_pos(la, F, std::min(total, ps.clusters), kVarF32, s));
  for (int i = 0; i < n; ++i) {
    const int rc = finish_job(jobs[i], L[i], jobs[i].B, s);
    if (rc) return rc;
  }
  return PTYCHO_OK;
}

}  // namespace

// One gradient step for several problems of the same window size.
int step_batch(const StepJob* jobs, int n, float2* slots, int nslots, long long slot_stride, const PosScratch* ps,
               unsigned* status, cudaStream_t s, int* tile_launches) {
  if (tile_launches) *tile_launches = 0;
  if (n < 1 || n > kMaxDesc) return perr(PTYCHO_EINVAL, "step_batch: 1..16 jobs");
  const EngineOps* ops = jobs[0].c->ops;
  bool pos = ps && ps->slots && ps->clusters > 0 && ops->has_variants;
  for (int i = 0; i < n; ++i) {
    const StepJob& J = jobs[i];
    ptycho_ctx* c = J.c;
    if (c->ops != ops || c->store) return perr(PTYCHO_EINVAL, "step_batch: mixed window sizes or stored waves");
    if (J.B < 1 || J.B > c->max_batch) return perr(PTYCHO_EINVAL, "step_batch: bad group size");
    if (c->g.K > (ps ? ps->kmodes : 0) || c->g.S > (ps ? ps->smax : 0) || c->g.wave_prec != PTYCHO_PREC_F32) pos = false;
  }
  if (pos) {
    if (tile_launches) *tile_launches = 1;
    return step_batch_pos(jobs, n, *ps, status, s);
  }
  if (tile_launches) *tile_launches = 2;
  LaunchArgs la{};
  la.nd = n;
  la.status = status;
  la.slots = reinterpret_cast<char*>(slots);
  la.slot_stride = slot_stride * 8;
  int total = 0;
  std::vector<Layout> L(n);
  std::vector<int> nl(n);
  for (int i = 0; i < n; ++i) {
    const StepJob& J = jobs[i];
    ptycho_ctx* c = J.c;
    if ((long long)c->g.S * c->NP * (c->g.wave_prec ? 4 : 8) > slot_stride * 8)
      return perr(PTYCHO_EINVAL, "step_batch: slot too small");
    L[i] = make_layout(c->g, c->max_batch, false, 0);
    CK(ops->probe_spectrum(J.P, reinterpret_cast<float2*>(c->arena + L[i].Phat), c->g.K, s));
    CK(cudaMemsetAsync(c->arena + L[i].gPhat, 0, (size_t)c->g.K * c->NP * 8, s));
    CK(cudaMemsetAsync(c->gO, 0, (size_t)c->g.S * c->g.H * c->g.W * 8, s));
    ProblemDesc d = base_desc(c, L[i], reinterpret_cast<const ptycho_c64*>(J.O), J.pos, J.idx, J.B, J.n_pos);
    d.gO = c->gO;
    d.item0 = total;
    total += J.B * c->g.K;
    la.d[i] = d;
  }
  la.total = total;
  CK(ops->forward(la, std::min(total, jobs[0].c->res_fwd), false, kVarF32, s));
  for (int i = 0; i < n; ++i) {
    const StepJob& J = jobs[i];
    ptycho_ctx* c = J.c;
    nl[i] = (int)std::min<long long>(kLossBlocks, ((long long)J.B * c->NP + 255) / 256);
    CK(ops->loss(la.d[i].A, J.Iexp, J.idx, J.n_pos, J.B, c->g.K, c->g.loss, (float)c->g.eps, (float)c->g.c,
                 reinterpret_cast<float*>(c->arena + L[i].w), reinterpret_cast<double*>(c->arena + L[i].partials),
                 nl[i], s));
  }
  CK(ops->adjoint(la, std::min(total, nslots), false, kVarF32, s));
  for (int i = 0; i < n; ++i) {
    const int rc = finish_job(jobs[i], L[i], nl[i], s);
    if (rc) return rc;
  }
  return PTYCHO_OK;
}

}  // namespace ptycho
