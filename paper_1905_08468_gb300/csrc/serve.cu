// Request server: continuous batching of MUFFIN deconvolutions.
//
// Requests (a PSF cube and a dirty cube of any side n and band count L,
// fixed (mu, gamma), an iteration count) are queued on submit.  Requests of
// one shape share a batched plan (a "pool", one per (n, L)); every pool
// advances on its own streams, independently of the others, a chunk of
// iterations at a time.  Each scheduling step, without waiting for the
// slowest pool:
//   1. collects the pools whose chunk has finished (an event per pool) and
//      retires their finished slots (the cube is copied to the request's
//      result and the slot is freed);
//   2. admits queued requests in arrival order (never overtaking the head of
//      the queue) while the voxels in slots stay under a cap, into a free
//      slot of an idle pool of their shape, creating a pool only when its
//      device footprint fits the server's HBM budget (idle pools of other
//      shapes are released first when memory is short);
//   3. launches the next chunk of every idle pool with active slots (all
//      slots of a pool in the same kernels; a slot never runs past its own
//      iteration count) on a stream whose priority follows the age of the
//      pool's oldest request: the oldest work gets the GPU first, as it
//      would one cube per launch in arrival order, and younger pools fill
//      the rest of the machine;
//   4. if nothing finished and nothing was launched, waits (briefly, by
//      polling) for a pool to finish its chunk.
// A slot's arithmetic does not depend on its neighbours, so a request's
// result is the same alone and in the mix.
#include <cuda_runtime.h>

#include <cmath>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "plan_internal.h"

using namespace muffin;

namespace {

struct Request {
  uint64_t id = 0;
  int n = 0, L = 0, iters = 0;
  double mu = 0, gamma = 0;
  std::vector<float> psf, dirty, result;
  int state = 0;            // 0 queued, 1 active, 2 done, 3 failed
  int pool = -1, slot = -1, done_iters = 0;
  muffin_status err = MUFFIN_OK;   // state 3: why (a non-finite input)
  std::string msg;
};

struct Pool {
  int n = 0, L = 0;
  muffin_plan plan = nullptr;
  std::vector<int64_t> slot_req;   // -1 = free
  cudaEvent_t done = nullptr;      // recorded after the chunk in flight
  bool busy = false;               // a chunk is in flight
  int run = 0;                     // iterations of that chunk
  cudaStream_t own_ws = nullptr;   // the plan's own work stream (lowest priority)
  cudaStream_t prio[2] = {nullptr, nullptr};   // highest and second priority
  int active() const {
    int a = 0;
    for (int64_t r : slot_req) a += r >= 0;
    return a;
  }
};

}  // namespace

struct muffin_server_s {
  muffin_server_params p{};
  cudaStream_t st = nullptr;
  size_t budget = 0, used = 0;
  uint64_t next_id = 1;
  std::deque<uint64_t> queue;
  std::map<uint64_t, Request> reqs;
  std::vector<Pool> pools;
};

namespace {

// slots per pool: max_batch, but no more than the active-work cap can fill
muffin_params pool_params(const muffin_server_s *S, int n, int L) {
  muffin_params p;
  muffin_params_default(&p, n, L);
  p.n_wavelets = S->p.n_wavelets;
  p.levels = S->p.levels;
  p.sigma = S->p.sigma;
  p.step_rule = S->p.step_rule;
  p.tau_safety = S->p.tau_safety;
  const size_t vox = (size_t)L * n * n;
  const size_t fit = std::max<size_t>(1, S->p.max_active_voxels / vox);
  p.batch = (int32_t)std::min<size_t>((size_t)S->p.max_batch, fit);
  return p;
}

void release_pool(muffin_server_s *S, size_t i) {
  Pool &pl = S->pools[i];
  if (pl.busy) cudaEventSynchronize(pl.done);
  if (pl.plan) {
    S->used -= muffin_plan_device_bytes(pl.plan);
    pl.plan->ws = pl.own_ws;          // the plan destroys its own stream
    muffin_plan_destroy(pl.plan);
  }
  for (cudaStream_t q : pl.prio)
    if (q) cudaStreamDestroy(q);
  if (pl.done) cudaEventDestroy(pl.done);
  S->pools.erase(S->pools.begin() + i);
  for (auto &kv : S->reqs)
    if (kv.second.pool > (int)i) kv.second.pool--;
}

// an idle pool for (n, L) with a free slot, creating one within the budget;
// -1: none now (every pool of the shape busy or full, or no memory)
int find_pool(muffin_server_s *S, int n, int L, muffin_status *err) {
  bool shape_has_room = false;
  for (size_t i = 0; i < S->pools.size(); ++i) {
    Pool &pl = S->pools[i];
    if (pl.n != n || pl.L != L) continue;
    for (int64_t r : pl.slot_req)
      if (r < 0) {
        if (!pl.busy) return (int)i;
        shape_has_room = true;
        break;
      }
  }
  // a busy pool of this shape will take the request at its chunk boundary
  if (shape_has_room) return -1;
  // no pool of this shape has a free slot: open another if it fits
  muffin_params p = pool_params(S, n, L);
  size_t need = 0;
  *err = muffin_plan_estimate_bytes(&p, &need);
  if (*err != MUFFIN_OK) return -1;
  // release idle pools of other shapes while memory is short
  for (size_t i = 0; i < S->pools.size() && S->used + need > S->budget;) {
    if (S->pools[i].active() == 0 && !S->pools[i].busy) release_pool(S, i);
    else ++i;
  }
  if (S->used + need > S->budget) return -1;
  Pool pl;
  pl.n = n; pl.L = L;
  *err = pi::create(&p, nullptr, nullptr, nullptr, S->st, &pl.plan);
  if (*err != MUFFIN_OK) return -1;
  const size_t got = muffin_plan_device_bytes(pl.plan);
  int lo = 0, hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl.done, cudaEventDisableTiming);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    e = cudaStreamCreateWithPriority(&pl.prio[k], cudaStreamNonBlocking,
                                     std::min(lo, hi + k) /* hi is the greatest */);
  if (e != cudaSuccess || S->used + got > S->budget) {  // (the estimate was short)
    for (cudaStream_t q : pl.prio)
      if (q) cudaStreamDestroy(q);
    if (pl.done) cudaEventDestroy(pl.done);
    muffin_plan_destroy(pl.plan);
    if (e != cudaSuccess) *err = fail(MUFFIN_ECUDA, "pool streams: %s", cudaGetErrorString(e));
    return -1;
  }
  pl.own_ws = pl.plan->ws;
  pl.slot_req.assign(p.batch, -1);
  S->used += got;
  S->pools.push_back(pl);
  return (int)S->pools.size() - 1;
}

size_t active_voxels(const muffin_server_s *S) {
  size_t active = 0;
  for (const auto &kv : S->reqs)
    if (kv.second.state == 1) active += (size_t)kv.second.L * kv.second.n * kv.second.n;
  return active;
}

// loads request r (inputs psf, dirty: host or device arrays) into a free
// slot of idle pool pi_; a non-finite input (MUFFIN_ENUMERIC, or EINVAL for a
// PSF whose spectrum is not finite) fails the request, not the server
muffin_status load_request(muffin_server_s *S, Request &r, int pi_, const float *psf,
                           const float *dirty) {
  Pool &pl = S->pools[pi_];
  int slot = 0;
  while (pl.slot_req[slot] >= 0) ++slot;
  muffin_plan P = pl.plan;
  muffin_status s = pi::enter(P);
  if (s == MUFFIN_OK) s = pi::load_psf(P, slot, slot + 1, psf);
  if (s == MUFFIN_OK) s = pi::load_dirty(P, slot, slot + 1, dirty);
  if (s == MUFFIN_OK) s = pi::reset_cubes(P, 0, slot, slot + 1, nullptr);
  if (s == MUFFIN_OK) s = pi::set_theta(P, slot, slot + 1, &r.mu, &r.gamma);
  std::vector<float>().swap(r.psf);     // inputs are on the device now (or rejected)
  std::vector<float>().swap(r.dirty);
  if (s == MUFFIN_ENUMERIC || s == MUFFIN_EINVAL) {
    r.state = 3; r.err = s; r.msg = muffin_last_error();
    return MUFFIN_OK;
  }
  if (s != MUFFIN_OK) return s;
  pl.slot_req[slot] = (int64_t)r.id;
  r.state = 1; r.pool = pi_; r.slot = slot; r.done_iters = 0;
  return MUFFIN_OK;
}

// admission in arrival order while the active work (voxels in slots) stays
// under the cap; the head of the queue is never overtaken
muffin_status admit(muffin_server_s *S, bool *admitted) {
  size_t active = active_voxels(S);
  for (auto it = S->queue.begin(); it != S->queue.end();) {
    Request &r = S->reqs[*it];
    const size_t vox = (size_t)r.L * r.n * r.n;
    if (active > 0 && active + vox > S->p.max_active_voxels) break;
    muffin_status err = MUFFIN_OK;
    const int pi_ = find_pool(S, r.n, r.L, &err);
    if (err != MUFFIN_OK) return err;
    if (pi_ < 0) break;
    muffin_status s = load_request(S, r, pi_, r.psf.data(), r.dirty.data());
    if (s != MUFFIN_OK) return s;
    if (r.state == 1) active += vox;
    *admitted = true;
    it = S->queue.erase(it);
  }
  return MUFFIN_OK;
}

// pools whose chunk has finished: account the iterations, retire finished slots
muffin_status collect(muffin_server_s *S, bool *progressed) {
  for (size_t i = 0; i < S->pools.size(); ++i) {
    Pool &pl = S->pools[i];
    if (!pl.busy) continue;
    const cudaError_t q = cudaEventQuery(pl.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return fail(MUFFIN_ECUDA, "pool chunk: %s", cudaGetErrorString(q));
    pl.busy = false;
    *progressed = true;
    bool fetched = false;
    for (size_t b = 0; b < pl.slot_req.size(); ++b) {
      const int64_t id = pl.slot_req[b];
      if (id < 0) continue;
      Request &r = S->reqs[(uint64_t)id];
      r.done_iters += pl.run;
      if (r.done_iters >= r.iters) {
        r.result.resize((size_t)r.L * r.n * r.n);
        muffin_status s = pi::fetch_x(pl.plan, (int)b, (int)b + 1, r.result.data());
        if (s != MUFFIN_OK) return s;
        fetched = true;
        r.state = 2;
        pl.slot_req[b] = -1;
      }
    }
    if (fetched) {
      muffin_status s = pi::leave(pl.plan, true);
      if (s != MUFFIN_OK) return s;
    }
  }
  return MUFFIN_OK;
}

// next chunk of every idle pool with active slots, on a stream whose
// priority follows the age (request id) of the pool's oldest request
muffin_status launch(muffin_server_s *S, bool *launched) {
  std::vector<std::pair<uint64_t, size_t>> order;
  for (size_t i = 0; i < S->pools.size(); ++i) {
    const Pool &pl = S->pools[i];
    uint64_t oldest = UINT64_MAX;
    for (int64_t r : pl.slot_req)
      if (r >= 0) oldest = std::min(oldest, (uint64_t)r);
    if (oldest != UINT64_MAX) order.push_back({oldest, i});
  }
  std::sort(order.begin(), order.end());
  for (size_t rank = 0; rank < order.size(); ++rank) {
    Pool &pl = S->pools[order[rank].second];
    if (pl.busy) continue;
    // the runs of consecutive slots that hold requests (free slots are not
    // computed; admission fills the lowest free slot first).  A pool that
    // is the only one with work while nothing is queued takes longer chunks
    // (fewer host round trips), up to 4x
    int run = (order.size() == 1 && S->queue.empty()) ? 4 * S->p.chunk : S->p.chunk;
    std::vector<std::pair<int, int>> runs;
    for (int b = 0; b < (int)pl.slot_req.size(); ++b)
      if (pl.slot_req[b] >= 0) {
        const Request &r = S->reqs[(uint64_t)pl.slot_req[b]];
        run = std::min(run, r.iters - r.done_iters);
        if (!runs.empty() && runs.back().second == b) runs.back().second = b + 1;
        else runs.push_back({b, b + 1});
      }
    if (runs.empty() || run <= 0) continue;
    muffin_plan P = pl.plan;
    P->ws = rank < 2 ? pl.prio[rank] : pl.own_ws;
    muffin_status s = pi::enter(P);
    if (s == MUFFIN_OK) s = pi::run_plain(P, run, runs);
    if (s != MUFFIN_OK) return s;
    MUFFIN_CK(cudaEventRecord(pl.done, P->ws));
    pl.busy = true;
    pl.run = run;
    *launched = true;
  }
  return MUFFIN_OK;
}

}  // namespace

extern "C" {

void muffin_server_params_default(muffin_server_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->hbm_budget_bytes = 0;
  p->max_batch = 8;
  p->n_wavelets = 8;
  p->levels = 3;
  p->sigma = 10.0;
  p->step_rule = 0;
  p->tau_safety = 0.99;
  p->chunk = 10;
  p->max_active_voxels = (size_t)3 << 24;
}

muffin_status muffin_server_create(const muffin_server_params *p, void *stream,
                                   muffin_server *out) {
  if (!p || !out) return fail(MUFFIN_EINVAL, "NULL argument");
  *out = nullptr;
  if (p->max_batch < 1 || p->chunk < 1 || p->max_active_voxels < 1)
    return fail(MUFFIN_EINVAL, "max_batch, chunk and max_active_voxels must be >= 1");
  muffin_server S = new (std::nothrow) muffin_server_s();
  if (!S) return fail(MUFFIN_ENOMEM, "host allocation failed");
  S->p = *p;
  S->st = static_cast<cudaStream_t>(stream);
  S->budget = p->hbm_budget_bytes;
  if (S->budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      delete S;
      return fail(MUFFIN_ECUDA, "cudaMemGetInfo failed (no device?)");
    }
    S->budget = fr / 10 * 8;
  }
  *out = S;
  return MUFFIN_OK;
}

void muffin_server_destroy(muffin_server S) {
  if (!S) return;
  while (!S->pools.empty()) release_pool(S, S->pools.size() - 1);
  delete S;
}

muffin_status muffin_serve_submit(muffin_server S, int32_t n, int32_t nbands,
                                  const float *psf, const float *dirty, double mu,
                                  double gamma, int32_t iters, uint64_t *ticket) {
  if (!S || !psf || !dirty || !ticket) return fail(MUFFIN_EINVAL, "NULL argument");
  if (iters < 1) return fail(MUFFIN_EINVAL, "iters must be >= 1");
  if (!(mu >= 0) || !(gamma >= 0)) return fail(MUFFIN_EINVAL, "mu, gamma must be >= 0");
  muffin_params p = pool_params(S, n, nbands);
  size_t need = 0;
  muffin_status s = muffin_plan_estimate_bytes(&p, &need);
  if (s != MUFFIN_OK) return s;
  if (need > S->budget)
    return fail(MUFFIN_ENOMEM, "a %dx%dx%d pool needs %zu bytes > budget %zu", n, n, nbands,
                need, S->budget);
  Request r;
  r.id = S->next_id++;
  r.n = n; r.L = nbands; r.iters = iters; r.mu = mu; r.gamma = gamma;
  *ticket = r.id;
  // nothing queued ahead and an idle pool free (or creatable) within the
  // caps: admit at once, straight from the caller's arrays
  if (S->queue.empty()) {
    const size_t vox = (size_t)nbands * n * n, active = active_voxels(S);
    if (active == 0 || active + vox <= S->p.max_active_voxels) {
      muffin_status err = MUFFIN_OK;
      const int pi_ = find_pool(S, n, nbands, &err);
      if (err != MUFFIN_OK) return err;
      if (pi_ >= 0) {
        auto ins = S->reqs.emplace(r.id, std::move(r)).first;
        muffin_status ls = load_request(S, ins->second, pi_, psf, dirty);
        if (ls != MUFFIN_OK) S->reqs.erase(ins);
        return ls;
      }
    }
  }
  const size_t cnt = (size_t)nbands * n * n;
  r.psf.resize(cnt);
  r.dirty.resize(cnt);
  for (int k = 0; k < 2; ++k) {
    const float *src = k ? dirty : psf;
    float *dst = k ? r.dirty.data() : r.psf.data();
    if (is_device_ptr(src)) {
      cudaError_t e = cudaMemcpy(dst, src, cnt * sizeof(float), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return fail(MUFFIN_ECUDA, "copy of request input: %s", cudaGetErrorString(e));
    } else {
      std::memcpy(dst, src, cnt * sizeof(float));
    }
  }
  S->queue.push_back(r.id);
  S->reqs.emplace(r.id, std::move(r));
  return MUFFIN_OK;
}

muffin_status muffin_serve_step(muffin_server S, int32_t *active, int32_t *queued) {
  if (!S) return fail(MUFFIN_EINVAL, "server is NULL");
  // collect, admit, launch; when none of these happened while chunks are in
  // flight, wait for the first of them to finish and go again, so that
  // every step makes progress
  const auto t0 = std::chrono::steady_clock::now();
  for (int round = 0;; ++round) {
    bool progressed = false, admitted = false, launched = false;
    muffin_status s = collect(S, &progressed);
    if (s == MUFFIN_OK) s = admit(S, &admitted);
    if (s == MUFFIN_OK) s = launch(S, &launched);
    if (s != MUFFIN_OK) return s;
    if (progressed || admitted || launched || round > 0) break;
    bool any_busy = false;
    for (const Pool &pl : S->pools) any_busy |= pl.busy;
    if (!any_busy) break;
    // poll: spin for the first 200 us (a chunk boundary is often that
    // close), then yield between polls
    for (bool ready = false; !ready;) {
      for (const Pool &pl : S->pools)
        if (pl.busy && cudaEventQuery(pl.done) != cudaErrorNotReady) ready = true;
      if (ready) break;
      const auto dt = std::chrono::steady_clock::now() - t0;
      if (dt > std::chrono::seconds(60))
        return fail(MUFFIN_ETIMEOUT, "no pool finished its chunk within 60 s");
      if (dt > std::chrono::microseconds(200))
        std::this_thread::sleep_for(std::chrono::microseconds(10));
    }
  }
  if (active) {
    int a = 0;
    for (const Pool &pl : S->pools) a += pl.active();
    *active = a;
  }
  if (queued) *queued = (int32_t)S->queue.size();
  return MUFFIN_OK;
}

muffin_status muffin_serve_poll(muffin_server S, uint64_t ticket, int32_t *done,
                                float *x_out) {
  if (!S || !done) return fail(MUFFIN_EINVAL, "NULL argument");
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(MUFFIN_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  Request &r = it->second;
  if (r.state == 3) {             // rejected at admission: report and release
    *done = 1;
    const muffin_status e = r.err;
    const std::string m = r.msg;
    S->reqs.erase(it);
    return fail(e, "request %llu: %s", (unsigned long long)ticket, m.c_str());
  }
  *done = r.state == 2;
  if (!*done) return MUFFIN_OK;
  if (x_out) {
    const size_t bytes = r.result.size() * sizeof(float);
    if (is_device_ptr(x_out)) {
      cudaError_t e = cudaMemcpy(x_out, r.result.data(), bytes, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return fail(MUFFIN_ECUDA, "copy of result: %s", cudaGetErrorString(e));
    } else {
      std::memcpy(x_out, r.result.data(), bytes);
    }
    S->reqs.erase(it);     // delivered
  }
  return MUFFIN_OK;
}

muffin_status muffin_server_stats(muffin_server S, size_t *device_bytes, int32_t *pools) {
  if (!S) return fail(MUFFIN_EINVAL, "server is NULL");
  if (device_bytes) *device_bytes = S->used;
  if (pools) *pools = (int32_t)S->pools.size();
  return MUFFIN_OK;
}

}  // extern "C"
