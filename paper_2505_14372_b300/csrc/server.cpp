// In-process continuous-batching server (arXiv 2505.14372 §2.3: clients
// submit reconstruction jobs, workers run them and report state; here one
// worker thread drives one GPU).
//
// Requests from datasets of different shapes are admitted against an HBM
// budget as memory and slots free up; each admitted request keeps its object,
// probe, Adam moments, positions and patterns resident.  Every scheduling
// tick issues one gradient step (one group) for each active request: the
// requests that share a window size ride in one position-major loss +
// adjoint launch (their positions from several problem descriptors; when
// the budget has no room for its scratch, in one forward and one
// recomputing adjoint launch instead), and the window-size classes run on
// their own streams, so their work overlaps on the device.  Per-iteration
// latency is measured with CUDA events.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "errors.h"
#include "internal.h"
#include "launch.h"
#include "ptycho.h"

using ptycho::StepJob;

namespace {

constexpr int kMaxSlices = 32;       // slot scratch is sized for this many slices
constexpr int kPosModes = 8;         // position-major scratch holds this many modes
constexpr int kMaxInflight = 2;      // ticks queued per stream
constexpr int kClasses = 4;          // window sizes 64, 128, 192, 256
const int kN[kClasses] = {64, 128, 192, 256};

int class_of(int N) {
  for (int i = 0; i < kClasses; ++i)
    if (kN[i] == N) return i;
  return -1;
}

struct Request {
  uint64_t ticket = 0;
  ptycho_request req{};
  std::vector<double> dz;
  std::vector<float> pos, Iexp;
  std::vector<ptycho_c64> O0, P0;
  int cls = 0;
  int state = PTYCHO_REQ_QUEUED;
  int error = 0;
  size_t need = 0;
  double submit_ms = 0, start_ms = -1, finish_ms = -1;
  // device state while running
  ptycho_ctx* ctx = nullptr;
  float2 *O = nullptr, *P = nullptr, *mO = nullptr, *mP = nullptr;
  float *vO = nullptr, *vP = nullptr, *dpos = nullptr, *dI = nullptr;
  int* didx = nullptr;           // 2 x n_pos (iteration parity)
  double* dstats = nullptr;      // [total steps][2]
  std::vector<int32_t> perm;
  int groups = 0, group = 0, iteration = 0, steps_issued = 0, steps_done = 0, total_steps = 0;
  int64_t t = 0;
  cudaEvent_t start_ev = nullptr;
  cudaEvent_t last_iter_ev = nullptr;  // not owned: the tick event that closed the previous iteration
  double last_iter_ms = -1;
  int iterations_done = 0;
  double last_loss = 0;
  // stopping: non-zero once the request is to end without finishing
  // (PTYCHO_ECANCELED, PTYCHO_ENONFINITE); no new steps are issued for it,
  // and it fails once none of its ticks is in flight
  int stop_code = 0;
  int inflight = 0;                 // ticks in flight that include it
  double* iter_loss = nullptr;      // pinned host [iterations]: loss of each iteration's last step

  // results
  std::vector<ptycho_c64> O_out, P_out;
  std::vector<double> loss_out, step_ms, iter_ms;
};

struct Tick {
  cudaEvent_t ev = nullptr;
  std::vector<std::pair<Request*, bool>> who;  // (request, closes an iteration)
  int positions = 0;
};

struct Class {
  cudaStream_t stream = nullptr;
  float2* slots = nullptr;
  int nslots = 0;
  long long stride = 0;
  size_t bytes = 0;
  // scratch of the position-major step (null when the budget has no room
  // for it: the class then runs the forward + recomputing adjoint launches)
  char* pos_mem = nullptr;
  size_t pos_bytes = 0;
  ptycho::PosScratch ps;
  std::deque<Tick> inflight;
  cudaEvent_t last_ev = nullptr;  // end of the previous tick on this stream
  size_t rr = 0;                  // round-robin cursor
};

double host_ms(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

size_t request_bytes(const ptycho_request& q) {
  const ptycho_geom& g = q.geom;
  const size_t nO = (size_t)g.S * g.H * g.W, NP = (size_t)g.h * g.w, nP = (size_t)g.K * NP;
  ptycho_geom gg = g;
  gg.waves = PTYCHO_WAVES_RECOMPUTE;
  // scratch of one step without own slots: the store-free layout is what
  // ptycho_scratch_bytes reports for RECOMPUTE minus the slot part
  const size_t B = (size_t)q.batch;
  const size_t scratch = nP * 8 * 2 + B * g.K * NP * 8 + B * NP * 4 * 2 + B * 8 + 64 * 1024;
  const size_t grads = nO * 8 + nP * 8 + (g.S > 1 ? (size_t)(g.S - 1) * g.h * 8 : 0);
  const size_t state = nO * 20 + nP * 20;
  const size_t data = (size_t)q.n_pos * 8 + (size_t)q.n_pos * NP * 4 + (size_t)q.n_pos * 8;
  const size_t groups = ((size_t)q.n_pos + B - 1) / B;
  const size_t stats = groups * (size_t)q.iterations * 16;
  return scratch + grads + state + data + stats;
}

}  // namespace

struct ptycho_server {
  size_t budget = 0;
  int max_active = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::map<uint64_t, std::unique_ptr<Request>> all;
  std::vector<Request*> active;
  size_t admitted_bytes = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  std::chrono::steady_clock::time_point host0;
  cudaEvent_t t0 = nullptr;  // device time origin (recorded at creation)
  size_t slot_bytes = 0;       // recompute scratch of the window classes in use
  Class cls[kClasses];
  unsigned* status = nullptr;
  // statistics
  int64_t n_submitted = 0, n_admitted = 0, n_finished = 0, n_failed = 0, n_launches = 0;
  double positions_done = 0, first_start_ms = -1, last_end_ms = -1;
  std::vector<double> iter_lat;
  double stall_ms = 0;  // host-side fault injection: the worker sleeps this long before its next tick

  void run();
  int admit(Request* r);
  void release_device(Request* r);
  void fail(Request* r, int code);
  bool retire_ticks();
  bool issue_ticks();
  void finish(Request* r);
};

void ptycho_server::release_device(Request* r) {
  if (r->ctx) ptycho_destroy(r->ctx);
  r->ctx = nullptr;
  for (void* p : {(void*)r->O, (void*)r->P, (void*)r->mO, (void*)r->mP, (void*)r->vO, (void*)r->vP,
                  (void*)r->dpos, (void*)r->dI, (void*)r->didx, (void*)r->dstats})
    cudaFree(p);
  r->O = r->P = r->mO = r->mP = nullptr;
  r->vO = r->vP = r->dpos = r->dI = nullptr;
  r->didx = nullptr;
  r->dstats = nullptr;
  if (r->start_ev) cudaEventDestroy(r->start_ev);
  r->start_ev = nullptr;
  if (r->iter_loss) cudaFreeHost(r->iter_loss);
  r->iter_loss = nullptr;
}

void ptycho_server::fail(Request* r, int code) {
  r->state = PTYCHO_REQ_FAILED;
  r->error = code;
  r->finish_ms = host_ms(host0);
  release_device(r);
  admitted_bytes -= r->need;
  active.erase(std::remove(active.begin(), active.end(), r), active.end());
  ++n_failed;
}

// Allocates and uploads one request's resident state (worker thread).
int ptycho_server::admit(Request* r) {
  const ptycho_geom& g = r->req.geom;
  Class& C = cls[r->cls];
  if (!C.stream) {
    if (cudaStreamCreateWithFlags(&C.stream, cudaStreamNonBlocking) != cudaSuccess) return PTYCHO_ECUDA;
    C.nslots = ptycho::resident_slots(g.h);
    C.stride = (long long)kMaxSlices * g.h * g.w;
    C.bytes = (size_t)C.nslots * C.stride * 8;
    if (cudaMalloc(&C.slots, C.bytes) != cudaSuccess) {
      cudaGetLastError();
      C.slots = nullptr;
      C.bytes = 0;
      return PTYCHO_ENOMEM;
    }
    slot_bytes += C.bytes;
    const size_t pb = ptycho::pos_scratch_bytes(g.h, kPosModes, kMaxSlices);
    if (admitted_bytes + slot_bytes + pb <= budget && cudaMalloc(&C.pos_mem, pb) == cudaSuccess) {
      C.pos_bytes = pb;
      C.ps = ptycho::pos_scratch_at(C.pos_mem, g.h, kPosModes, kMaxSlices);
      slot_bytes += pb;
      // the launches' work queue starts empty (each launch leaves it so)
      if (cudaMemsetAsync(C.ps.queue, 0, 2 * sizeof(unsigned), C.stream) != cudaSuccess) {
        cudaGetLastError();
        return PTYCHO_ECUDA;
      }
    } else {
      cudaGetLastError();
      C.pos_mem = nullptr;
    }
  }
  ptycho_geom gg = g;
  gg.dz = r->dz.empty() ? nullptr : r->dz.data();
  int rc = ptycho::ctx_create_shared_slots(&gg, r->req.batch, &r->ctx);
  if (rc) return rc;
  const size_t nO = (size_t)g.S * g.H * g.W, NP = (size_t)g.h * g.w, nP = (size_t)g.K * NP;
  const int n = r->req.n_pos;
  r->groups = (n + r->req.batch - 1) / r->req.batch;
  r->total_steps = r->groups * r->req.iterations;
  bool ok = cudaMalloc(&r->O, nO * 8) == cudaSuccess && cudaMalloc(&r->mO, nO * 8) == cudaSuccess &&
            cudaMalloc(&r->vO, nO * 4) == cudaSuccess && cudaMalloc(&r->P, nP * 8) == cudaSuccess &&
            cudaMalloc(&r->mP, nP * 8) == cudaSuccess && cudaMalloc(&r->vP, nP * 4) == cudaSuccess &&
            cudaMalloc(&r->dpos, (size_t)n * 8) == cudaSuccess && cudaMalloc(&r->dI, (size_t)n * NP * 4) == cudaSuccess &&
            cudaMalloc(&r->didx, (size_t)n * 8) == cudaSuccess &&
            cudaMalloc(&r->dstats, (size_t)r->total_steps * 16) == cudaSuccess &&
            cudaMallocHost(&r->iter_loss, (size_t)r->req.iterations * 8) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return PTYCHO_ENOMEM;
  }
  cudaStream_t s = C.stream;
  ok = cudaMemcpyAsync(r->O, r->O0.data(), nO * 8, cudaMemcpyHostToDevice, s) == cudaSuccess &&
       cudaMemcpyAsync(r->P, r->P0.data(), nP * 8, cudaMemcpyHostToDevice, s) == cudaSuccess &&
       cudaMemcpyAsync(r->dpos, r->pos.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s) == cudaSuccess &&
       cudaMemcpyAsync(r->dI, r->Iexp.data(), (size_t)n * NP * 4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
       cudaMemsetAsync(r->mO, 0, nO * 8, s) == cudaSuccess && cudaMemsetAsync(r->vO, 0, nO * 4, s) == cudaSuccess &&
       cudaMemsetAsync(r->mP, 0, nP * 8, s) == cudaSuccess && cudaMemsetAsync(r->vP, 0, nP * 4, s) == cudaSuccess &&
       cudaEventCreate(&r->start_ev) == cudaSuccess && cudaEventRecord(r->start_ev, s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return PTYCHO_ECUDA;
  }
  // the host copies of the data are no longer needed
  std::vector<float>().swap(r->Iexp);
  std::vector<ptycho_c64>().swap(r->O0);
  r->perm.resize(n);
  return PTYCHO_OK;
}

void ptycho_server::finish(Request* r) {
  const ptycho_geom& g = r->req.geom;
  const size_t nO = (size_t)g.S * g.H * g.W, nP = (size_t)g.K * g.h * g.w;
  r->O_out.resize(nO);
  r->P_out.resize(nP);
  std::vector<double> st((size_t)r->total_steps * 2);
  cudaStream_t s = cls[r->cls].stream;
  bool ok = cudaMemcpyAsync(r->O_out.data(), r->O, nO * 8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaMemcpyAsync(r->P_out.data(), r->P, nP * 8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaMemcpyAsync(st.data(), r->dstats, st.size() * 8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    fail(r, PTYCHO_ECUDA);
    return;
  }
  r->loss_out.resize(r->total_steps);
  for (int i = 0; i < r->total_steps; ++i) r->loss_out[i] = st[2 * i];
  r->last_loss = r->total_steps ? st[2 * (r->total_steps - 1)] : 0.0;
  release_device(r);
  admitted_bytes -= r->need;
  active.erase(std::remove(active.begin(), active.end(), r), active.end());
  r->state = PTYCHO_REQ_DONE;
  r->finish_ms = host_ms(host0);
  ++n_finished;
}

// Retires completed ticks: per-iteration latency from device events.
bool ptycho_server::retire_ticks() {
  bool any = false;
  for (Class& C : cls) {
    while (!C.inflight.empty()) {
      Tick& tk = C.inflight.front();
      const cudaError_t q = cudaEventQuery(tk.ev);
      if (q == cudaErrorNotReady) break;
      for (auto& w : tk.who) w.first->inflight -= 1;
      if (q != cudaSuccess) {
        cudaGetLastError();
        for (auto& w : tk.who)
          if (w.first->state == PTYCHO_REQ_RUNNING) fail(w.first, PTYCHO_ECUDA);
      } else {
        float t_end = 0.f;
        cudaEventElapsedTime(&t_end, t0, tk.ev);
        last_end_ms = std::max(last_end_ms, (double)t_end);
        positions_done += tk.positions;
        for (auto& w : tk.who) {
          Request* r = w.first;
          if (r->state != PTYCHO_REQ_RUNNING) continue;
          r->steps_done += 1;
          if (w.second) {
            // the loss of the iteration's last step (copied after it): a
            // non-finite value ends the request (diverged, or data the
            // submit checks could not see through)
            if (!std::isfinite(r->iter_loss[r->iterations_done]) && !r->stop_code) r->stop_code = PTYCHO_ENONFINITE;
            double t_prev = r->last_iter_ms;
            if (t_prev < 0) {
              float ts = 0.f;
              cudaEventElapsedTime(&ts, t0, r->start_ev);
              t_prev = ts;
            }
            r->iter_ms.push_back(t_end - t_prev);
            iter_lat.push_back(t_end - t_prev);
            r->last_iter_ms = t_end;
            r->iterations_done += 1;
          }
        }
      }
      cudaEventDestroy(tk.ev);
      C.inflight.pop_front();
      any = true;
    }
  }
  for (Request* r : std::vector<Request*>(active)) {
    if (r->state != PTYCHO_REQ_RUNNING) continue;
    if (r->stop_code && r->inflight == 0) {  // nothing of it left on the device
      fail(r, r->stop_code);
      any = true;
    } else if (!r->stop_code && r->steps_done == r->total_steps) {
      finish(r);
      any = true;
    }
  }
  return any;
}

// Issues one step for every active request with work left, batched per
// window size (at most 16 problems per launch).
bool ptycho_server::issue_ticks() {
  bool any = false;
  for (int k = 0; k < kClasses; ++k) {
    Class& C = cls[k];
    if (!C.stream || (int)C.inflight.size() >= kMaxInflight) continue;
    std::vector<Request*> mine;
    for (Request* r : active)
      if (r->cls == k && r->state == PTYCHO_REQ_RUNNING && !r->stop_code && r->steps_issued < r->total_steps)
        mine.push_back(r);
    if (mine.empty()) continue;
    if (mine.size() > (size_t)ptycho::kMaxDesc) {
      std::rotate(mine.begin(), mine.begin() + (C.rr % mine.size()), mine.end());
      mine.resize(ptycho::kMaxDesc);
      C.rr += ptycho::kMaxDesc;
    }
    std::vector<StepJob> jobs;
    Tick tk;
    std::vector<std::pair<double*, const double*>> loss_copies;  // (pinned host, device) per closed iteration
    for (Request* r : mine) {
      const int n = r->req.n_pos, B = r->req.batch;
      if (r->group == 0) {
        ptycho_make_groups(n, B, r->req.seed, r->iteration, r->req.grouping, r->pos.data(), r->perm.data());
        int* dst = r->didx + (size_t)(r->iteration & 1) * n;
        if (cudaMemcpyAsync(dst, r->perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, C.stream) != cudaSuccess) {
          cudaGetLastError();
          fail(r, PTYCHO_ECUDA);
          continue;
        }
      }
      StepJob J{};
      J.c = r->ctx;
      J.O = r->O;
      J.P = r->P;
      J.mO = r->mO;
      J.vO = r->vO;
      J.mP = r->mP;
      J.vP = r->vP;
      J.t = ++r->t;
      J.opt = r->req.opt;
      J.pos = r->dpos;
      J.Iexp = r->dI;
      J.n_pos = n;
      J.idx = r->didx + (size_t)(r->iteration & 1) * n + (size_t)r->group * B;
      J.B = std::min(B, n - r->group * B);
      J.stats = r->dstats + 2 * (size_t)r->steps_issued;
      jobs.push_back(J);
      tk.positions += J.B;
      bool closes = false;
      r->steps_issued += 1;
      if (++r->group == r->groups) {
        loss_copies.push_back({r->iter_loss + r->iteration, J.stats});
        r->group = 0;
        r->iteration += 1;
        closes = true;
      }
      tk.who.push_back({r, closes});
    }
    if (jobs.empty()) continue;
    int tl = 0;
    char rn[64];
    std::snprintf(rn, sizeof rn, "serve tick: window %d, %d jobs", mine.front()->req.geom.h, (int)jobs.size());
    ptycho::Range range(rn);
    int rc = ptycho::step_batch(jobs.data(), (int)jobs.size(), C.slots, C.nslots, C.stride,
                                C.pos_mem ? &C.ps : nullptr, status, C.stream, &tl);
    for (const auto& lc : loss_copies)
      if (rc == PTYCHO_OK && cudaMemcpyAsync(lc.first, lc.second, sizeof(double), cudaMemcpyDeviceToHost, C.stream) !=
                                 cudaSuccess)
        rc = PTYCHO_ECUDA;
    if (rc == PTYCHO_OK && cudaEventCreate(&tk.ev) == cudaSuccess && cudaEventRecord(tk.ev, C.stream) == cudaSuccess) {
      for (auto& w : tk.who) w.first->inflight += 1;
      C.inflight.push_back(tk);
      n_launches += tl;
      any = true;
    } else {
      cudaGetLastError();
      for (auto& w : tk.who) fail(w.first, rc ? rc : PTYCHO_ECUDA);
    }
  }
  return any;
}

void ptycho_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    if (stall_ms > 0) {  // injected stall (tests of the clients' time-outs)
      const double ms = stall_ms;
      stall_ms = 0;
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds((long long)(ms * 1e3)));
      lk.lock();
      continue;
    }
    // admission: first come, first served, against slots and the HBM budget
    while (!queue.empty() && (int)active.size() < max_active) {
      Request* r = queue.front();
      const size_t slot = cls[r->cls].stream ? 0 : (size_t)ptycho::resident_slots(r->req.geom.h) * kMaxSlices *
                                                      r->req.geom.h * r->req.geom.w * 8;
      if (admitted_bytes + slot_bytes + r->need + slot > budget) break;
      queue.pop_front();
      admitted_bytes += r->need;
      active.push_back(r);
      r->state = PTYCHO_REQ_ADMITTING;
      lk.unlock();  // allocation and upload can take a while: do not block submit/poll
      const int rc = admit(r);
      lk.lock();
      if (rc) {
        fail(r, rc);
      } else {
        r->state = PTYCHO_REQ_RUNNING;
        r->start_ms = host_ms(host0);
        if (first_start_ms < 0) first_start_ms = r->start_ms;
        ++n_admitted;
      }
      if (stop) break;
    }
    bool progressed = retire_ticks();
    progressed |= issue_ticks();
    if (progressed) {
      cv.notify_all();
      continue;
    }
    // nothing to do right now: wait for the oldest tick or for a submit
    cudaEvent_t wait_ev = nullptr;
    for (Class& C : cls)
      if (!C.inflight.empty()) {
        wait_ev = C.inflight.front().ev;
        break;
      }
    if (wait_ev) {
      lk.unlock();
      cudaEventSynchronize(wait_ev);
      lk.lock();
    } else {
      cv.wait_for(lk, std::chrono::milliseconds(2));
    }
  }
}

extern "C" {

int ptycho_server_create(size_t hbm_budget_bytes, int32_t max_active, ptycho_server** out) {
  if (!out) return perr(PTYCHO_EINVAL, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes == 0 || max_active < 1) return perr(PTYCHO_EINVAL, "budget and max_active must be > 0");
  auto* s = new ptycho_server();
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  if (cudaGetDevice(&s->device) != cudaSuccess || cudaEventCreate(&s->t0) != cudaSuccess ||
      cudaMalloc(&s->status, sizeof(unsigned)) != cudaSuccess || cudaMemset(s->status, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaEventRecord(s->t0, 0) != cudaSuccess || cudaEventSynchronize(s->t0) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return perr(PTYCHO_ECUDA, "server: CUDA device setup failed");
  }
  s->host0 = std::chrono::steady_clock::now();
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return PTYCHO_OK;
}

int ptycho_server_destroy(ptycho_server* s) {
  if (!s) return PTYCHO_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  s->worker.join();
  cudaSetDevice(s->device);
  for (Class& C : s->cls) {
    if (C.stream) cudaStreamSynchronize(C.stream);
    for (Tick& t : C.inflight) cudaEventDestroy(t.ev);
    C.inflight.clear();
    cudaFree(C.slots);
    cudaFree(C.pos_mem);
    if (C.stream) cudaStreamDestroy(C.stream);
  }
  for (auto& kv : s->all) s->release_device(kv.second.get());
  cudaFree(s->status);
  cudaEventDestroy(s->t0);
  delete s;
  return PTYCHO_OK;
}

int ptycho_submit(ptycho_server* s, const ptycho_request* q, uint64_t* ticket) {
  if (!s || !q || !ticket) return perr(PTYCHO_EINVAL, "NULL argument");
  const ptycho_geom& g = q->geom;
  if (g.h != g.w || class_of(g.h) < 0) return perr(PTYCHO_EINVAL, "window must be 64, 128, 192 or 256 square");
  if (g.S < 1 || g.S > kMaxSlices) return perr(PTYCHO_EINVAL, "served requests need 1 <= S <= 32");
  if (g.dft != PTYCHO_DFT_FFT) return perr(PTYCHO_EINVAL, "served requests use the FFT tile (dft = 0)");
  if (g.K < 1 || g.H < g.h || g.W < g.w || (g.S > 1 && !g.dz)) return perr(PTYCHO_EINVAL, "bad geometry");
  if (q->n_pos < 1 || !q->pos || !q->I_exp || !q->P_init || q->iterations < 1 || q->batch < 1)
    return perr(PTYCHO_EINVAL, "bad request (positions, patterns, probe, iterations, batch)");
  if (q->grouping != 0 && q->grouping != 1) return perr(PTYCHO_EINVAL, "grouping must be 0 or 1");
  if ((q->opt.reg_obj_tv != 0.f || q->opt.reg_obj_layers_tv != 0.f) && !(q->opt.reg_tv_eps > 0.f))
    return perr(PTYCHO_EINVAL, "TV regularisers need reg_tv_eps > 0");
  if (g.wave_prec != PTYCHO_PREC_F32) return perr(PTYCHO_EINVAL, "served requests keep FP32 entry waves");
  if (g.deterministic) return perr(PTYCHO_EINVAL, "served requests use the atomic gradient sums (deterministic = 0)");
  if (int rc = ptycho::validate_geom(&g)) return rc;  // the rest of the geometry, as ptycho_create checks it
  // non-finite data would turn the whole reconstruction into NaN: refuse it
  // here, with the first offending index
  auto first_nonfinite = [](const float* a, size_t n) -> long long {
    for (size_t i = 0; i < n; ++i)
      if (!std::isfinite(a[i])) return (long long)i;
    return -1;
  };
  const size_t NPq = (size_t)g.h * g.w;
  if (long long i = first_nonfinite(q->pos, 2 * (size_t)q->n_pos); i >= 0)
    return perr(PTYCHO_EINVAL, "scan position " + std::to_string(i / 2) + " is not finite");
  if (long long i = first_nonfinite(q->I_exp, (size_t)q->n_pos * NPq); i >= 0)
    return perr(PTYCHO_EINVAL, "pattern " + std::to_string(i / (long long)NPq) + " holds a non-finite value");
  if (long long i = first_nonfinite(&q->P_init[0].re, 2 * (size_t)g.K * NPq); i >= 0)
    return perr(PTYCHO_EINVAL, "probe mode " + std::to_string(i / (2 * (long long)NPq)) + " holds a non-finite value");
  if (q->O_init)
    if (long long i = first_nonfinite(&q->O_init[0].re, 2 * (size_t)g.S * g.H * g.W); i >= 0)
      return perr(PTYCHO_EINVAL, "object slice " + std::to_string(i / (2LL * g.H * g.W)) + " holds a non-finite value");
  for (int j = 0; j < q->n_pos; ++j) {
    const double y = std::floor((double)q->pos[2 * j] + 0.5), x = std::floor((double)q->pos[2 * j + 1] + 0.5);
    if (!(y >= 0 && x >= 0 && y + g.h <= g.H && x + g.w <= g.W))
      return perr(PTYCHO_EOUTOFBOUNDS, "scan position " + std::to_string(j) + " leaves the object");
  }
  auto r = std::make_unique<Request>();
  r->req = *q;
  r->cls = class_of(g.h);
  r->need = request_bytes(*q);
  const size_t slot = (size_t)ptycho::resident_slots(g.h) * kMaxSlices * g.h * g.w * 8;
  if (r->need + slot > s->budget)
    return perr(PTYCHO_ENOMEM, "request needs " + std::to_string(r->need + slot) + " bytes, budget is " +
                                   std::to_string(s->budget));
  const size_t nO = (size_t)g.S * g.H * g.W, NP = (size_t)g.h * g.w;
  r->dz.assign(g.dz ? g.dz : nullptr, g.dz ? g.dz + std::max(g.S - 1, 0) : nullptr);
  r->pos.assign(q->pos, q->pos + 2 * (size_t)q->n_pos);
  r->Iexp.assign(q->I_exp, q->I_exp + (size_t)q->n_pos * NP);
  r->P0.assign(q->P_init, q->P_init + (size_t)g.K * NP);
  if (q->O_init) r->O0.assign(q->O_init, q->O_init + nO);
  else r->O0.assign(nO, ptycho_c64{1.0f, 0.0f});
  r->req.geom.dz = nullptr;
  r->req.pos = r->req.I_exp = nullptr;
  r->req.O_init = r->req.P_init = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  r->ticket = s->next_ticket++;
  r->submit_ms = host_ms(s->host0);
  *ticket = r->ticket;
  s->queue.push_back(r.get());
  s->all[r->ticket] = std::move(r);
  ++s->n_submitted;
  s->cv.notify_all();
  return PTYCHO_OK;
}

int ptycho_poll(ptycho_server* s, uint64_t ticket, ptycho_status* st, ptycho_result* res) {
  if (!s) return perr(PTYCHO_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return perr(PTYCHO_ENOTFOUND, "unknown ticket");
  Request* r = it->second.get();
  if (st) {
    st->state = r->state;
    st->iterations_done = r->iterations_done;
    st->error = r->error;
    st->last_loss = r->last_loss;
    st->submit_ms = r->submit_ms;
    st->start_ms = r->start_ms;
    st->finish_ms = r->finish_ms;
  }
  if (res) {
    std::memset(res, 0, sizeof(*res));
    if (r->state == PTYCHO_REQ_DONE) {
      res->O = r->O_out.data();
      res->P = r->P_out.data();
      res->loss = r->loss_out.data();
      res->n_loss = (int32_t)r->loss_out.size();
      res->step_ms = r->iter_ms.data();
      res->n_step = (int32_t)r->iter_ms.size();
    }
  }
  return PTYCHO_OK;
}

int ptycho_wait(ptycho_server* s, uint64_t ticket, double timeout_ms) {
  if (!s) return perr(PTYCHO_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds((long long)(timeout_ms * 1e3));
  for (;;) {
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return perr(PTYCHO_ENOTFOUND, "unknown ticket");
    const int st = it->second->state;
    if (st == PTYCHO_REQ_DONE) return PTYCHO_OK;
    if (st == PTYCHO_REQ_FAILED) return perr(it->second->error ? it->second->error : PTYCHO_ECUDA, "request failed");
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto it2 = s->all.find(ticket);
      if (it2 != s->all.end() && it2->second->state == PTYCHO_REQ_DONE) return PTYCHO_OK;
      return perr(PTYCHO_ETIMEDOUT, "request not finished before the timeout");
    }
  }
}

int ptycho_cancel(ptycho_server* s, uint64_t ticket) {
  if (!s) return perr(PTYCHO_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return perr(PTYCHO_ENOTFOUND, "unknown ticket");
  Request* r = it->second.get();
  if (r->state == PTYCHO_REQ_QUEUED) {  // never admitted: nothing on the device
    s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), r), s->queue.end());
    r->state = PTYCHO_REQ_FAILED;
    r->error = PTYCHO_ECANCELED;
    r->finish_ms = host_ms(s->host0);
    ++s->n_failed;
  } else if (r->state == PTYCHO_REQ_ADMITTING || r->state == PTYCHO_REQ_RUNNING) {
    // the worker issues no further step and ends it once its ticks are done
    if (!r->stop_code) r->stop_code = PTYCHO_ECANCELED;
  }
  s->cv.notify_all();
  return PTYCHO_OK;
}

int ptycho_server_inject_stall(ptycho_server* s, double ms) {
  if (!s) return perr(PTYCHO_EINVAL, "server is NULL");
  if (!(ms >= 0) || !std::isfinite(ms)) return perr(PTYCHO_EINVAL, "stall must be finite and >= 0 ms");
  std::lock_guard<std::mutex> lk(s->mu);
  s->stall_ms = ms;
  s->cv.notify_all();
  return PTYCHO_OK;
}

int ptycho_release(ptycho_server* s, uint64_t ticket) {
  if (!s) return perr(PTYCHO_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return perr(PTYCHO_ENOTFOUND, "unknown ticket");
  const int st = it->second->state;
  if (st != PTYCHO_REQ_DONE && st != PTYCHO_REQ_FAILED) return perr(PTYCHO_EBUSY, "request still queued or running");
  s->all.erase(it);
  return PTYCHO_OK;
}

int ptycho_server_stats_get(ptycho_server* s, ptycho_server_stats* o) {
  if (!s || !o) return perr(PTYCHO_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  o->submitted = s->n_submitted;
  o->admitted = s->n_admitted;
  o->finished = s->n_finished;
  o->failed = s->n_failed;
  o->queue_depth = (int64_t)s->queue.size();
  o->admitted_bytes = s->admitted_bytes + s->slot_bytes;
  o->budget_bytes = s->budget;
  o->launches = s->n_launches;
  const double busy = s->last_end_ms;  // device ms since the first tick
  o->positions_per_s = busy > 0 ? s->positions_done / (busy / 1e3) : 0.0;
  std::vector<double> v = s->iter_lat;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) {  // nearest-rank percentile
    if (v.empty()) return 0.0;
    const size_t rank = std::max<size_t>(1, (size_t)std::ceil(p * (double)v.size()));
    return v[std::min(rank, v.size()) - 1];
  };
  o->p50_iter_ms = pct(0.50);
  o->p99_iter_ms = pct(0.99);
  return PTYCHO_OK;
}

}  // extern "C"
