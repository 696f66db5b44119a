// Request server: continuous batching of MUFFIN deconvolutions.
//
// Requests (a PSF cube and a dirty cube of any side n and band count L,
// fixed (mu, gamma), an iteration count) are queued on submit.  Every
// scheduling step
//   1. admits queued requests in arrival order (never overtaking the head of
//      the queue) while the voxels in slots stay under a cap, into free slots
//      of a batched plan of their shape (one "pool" per (n, L)), creating a
//      pool only when its device footprint fits the server's HBM budget (idle
//      pools of other shapes are released first when memory is short);
//   2. advances every pool with active slots by up to `chunk` iterations in
//      shared launches (all slots of a pool run in the same kernels; a slot
//      never runs past its own iteration count);
//   3. retires finished slots: their cube is copied to the request's result
//      and the slot is freed for the next request.
// A slot's arithmetic does not depend on its neighbours, so a request's
// result is the same alone and in the mix.
#include <cuda_runtime.h>

#include <cmath>

#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "plan_internal.h"

using namespace muffin;

namespace {

struct Request {
  uint64_t id = 0;
  int n = 0, L = 0, iters = 0;
  double mu = 0, gamma = 0;
  std::vector<float> psf, dirty, result;
  int state = 0;            // 0 queued, 1 active, 2 done
  int pool = -1, slot = -1, done_iters = 0;
};

struct Pool {
  int n = 0, L = 0;
  muffin_plan plan = nullptr;
  std::vector<int64_t> slot_req;   // -1 = free
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

muffin_params pool_params(const muffin_server_s *S, int n, int L) {
  muffin_params p;
  muffin_params_default(&p, n, L);
  p.n_wavelets = S->p.n_wavelets;
  p.levels = S->p.levels;
  p.sigma = S->p.sigma;
  p.step_rule = S->p.step_rule;
  p.tau_safety = S->p.tau_safety;
  p.batch = S->p.max_batch;
  return p;
}

void release_pool(muffin_server_s *S, size_t i) {
  Pool &pl = S->pools[i];
  if (pl.plan) {
    S->used -= muffin_plan_device_bytes(pl.plan);
    muffin_plan_destroy(pl.plan);
  }
  S->pools.erase(S->pools.begin() + i);
  for (auto &kv : S->reqs)
    if (kv.second.pool > (int)i) kv.second.pool--;
}

// a pool for (n, L) with a free slot, creating one within the budget; -1: none now
int find_pool(muffin_server_s *S, int n, int L, muffin_status *err) {
  for (size_t i = 0; i < S->pools.size(); ++i) {
    Pool &pl = S->pools[i];
    if (pl.n != n || pl.L != L) continue;
    for (int64_t r : pl.slot_req)
      if (r < 0) return (int)i;
  }
  // no pool of this shape has a free slot: open another if it fits
  muffin_params p = pool_params(S, n, L);
  size_t need = 0;
  *err = muffin_plan_estimate_bytes(&p, &need);
  if (*err != MUFFIN_OK) return -1;
  // release idle pools of other shapes while memory is short
  for (size_t i = 0; i < S->pools.size() && S->used + need > S->budget;) {
    if (S->pools[i].active() == 0) release_pool(S, i);
    else ++i;
  }
  if (S->used + need > S->budget) return -1;
  Pool pl;
  pl.n = n; pl.L = L;
  *err = pi::create(&p, nullptr, nullptr, nullptr, S->st, &pl.plan);
  if (*err != MUFFIN_OK) return -1;
  const size_t got = muffin_plan_device_bytes(pl.plan);
  if (S->used + got > S->budget) {      // the estimate was short: keep the budget
    muffin_plan_destroy(pl.plan);
    return -1;
  }
  pl.slot_req.assign(p.batch, -1);
  S->used += got;
  S->pools.push_back(pl);
  return (int)S->pools.size() - 1;
}

// admission in arrival order while the active work (voxels in slots) stays
// under the cap; the head of the queue is never overtaken
muffin_status admit(muffin_server_s *S) {
  size_t active = 0;
  for (const auto &kv : S->reqs)
    if (kv.second.state == 1) active += (size_t)kv.second.L * kv.second.n * kv.second.n;
  for (auto it = S->queue.begin(); it != S->queue.end();) {
    Request &r = S->reqs[*it];
    const size_t vox = (size_t)r.L * r.n * r.n;
    if (active > 0 && active + vox > S->p.max_active_voxels) break;
    muffin_status err = MUFFIN_OK;
    const int pi_ = find_pool(S, r.n, r.L, &err);
    if (err != MUFFIN_OK) return err;
    if (pi_ < 0) break;
    Pool &pl = S->pools[pi_];
    int slot = 0;
    while (pl.slot_req[slot] >= 0) ++slot;
    muffin_plan P = pl.plan;
    muffin_status s = pi::enter(P);
    if (s == MUFFIN_OK) s = pi::load_psf(P, slot, slot + 1, r.psf.data());
    if (s == MUFFIN_OK) s = pi::load_dirty(P, slot, slot + 1, r.dirty.data());
    if (s == MUFFIN_OK) s = pi::reset_cubes(P, 0, slot, slot + 1, nullptr);
    if (s == MUFFIN_OK) s = pi::set_theta(P, slot, slot + 1, &r.mu, &r.gamma);
    if (s != MUFFIN_OK) return s;
    pl.slot_req[slot] = (int64_t)r.id;
    r.state = 1; r.pool = pi_; r.slot = slot; r.done_iters = 0;
    std::vector<float>().swap(r.psf);     // inputs are on the device now
    std::vector<float>().swap(r.dirty);
    active += vox;
    it = S->queue.erase(it);
  }
  return MUFFIN_OK;
}

muffin_status advance(muffin_server_s *S) {
  // launch every pool's chunk on its own stream first, so pools of different
  // shapes run concurrently on the device; then collect and synchronise
  std::vector<int> runs(S->pools.size(), 0);
  for (size_t i = 0; i < S->pools.size(); ++i) {
    Pool &pl = S->pools[i];
    int run = S->p.chunk, top = -1;
    for (size_t b = 0; b < pl.slot_req.size(); ++b)
      if (pl.slot_req[b] >= 0) {
        const Request &r = S->reqs[(uint64_t)pl.slot_req[b]];
        const int left = r.iters - r.done_iters;
        if (left < run) run = left;
        top = (int)b;
      }
    if (top < 0) continue;
    runs[i] = run;
    muffin_status s = pi::enter(pl.plan);
    if (s == MUFFIN_OK && run > 0) s = pi::run_plain(pl.plan, run, top + 1);
    if (s != MUFFIN_OK) return s;
  }
  for (size_t i = 0; i < S->pools.size(); ++i) {
    Pool &pl = S->pools[i];
    bool any = false;
    for (size_t b = 0; b < pl.slot_req.size(); ++b) {
      const int64_t id = pl.slot_req[b];
      if (id < 0) continue;
      any = true;
      Request &r = S->reqs[(uint64_t)id];
      r.done_iters += runs[i];
      if (r.done_iters >= r.iters) {
        r.result.resize((size_t)r.L * r.n * r.n);
        muffin_status s = pi::fetch_x(pl.plan, (int)b, (int)b + 1, r.result.data());
        if (s != MUFFIN_OK) return s;
        r.state = 2;
        pl.slot_req[b] = -1;
      }
    }
    if (any) {
      muffin_status s = pi::leave(pl.plan, true);
      if (s != MUFFIN_OK) return s;
    }
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
  for (size_t i = 0; i < cnt; ++i)
    if (!std::isfinite(r.dirty[i]) || !std::isfinite(r.psf[i]))
      return fail(MUFFIN_ENUMERIC, "request input has a NaN/Inf entry (index %zu)", i);
  *ticket = r.id;
  S->queue.push_back(r.id);
  S->reqs.emplace(r.id, std::move(r));
  return MUFFIN_OK;
}

muffin_status muffin_serve_step(muffin_server S, int32_t *active, int32_t *queued) {
  if (!S) return fail(MUFFIN_EINVAL, "server is NULL");
  muffin_status s = admit(S);
  if (s == MUFFIN_OK) s = advance(S);
  if (s != MUFFIN_OK) return s;
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
