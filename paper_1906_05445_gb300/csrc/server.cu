// server.cu -- a native serving engine over the C ABI: solves submitted as
// they arrive are admitted by their device-memory footprint and advanced
// together as an lbm_batch (continuous batching), each retired when its
// velocity residual falls below the tolerance.  The worker thread is the only
// user of the contexts and the batch; submit/poll/wait only touch the request
// table under the mutex.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/lbm.h"

struct lbm_server {
  int device = 0;
  size_t budget = 0;
  double tol = 1e-6;
  int check_every = 200;
  int max_steps = 200000;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  struct Req {
    lbm_request r;
    lbm_result res;
    std::vector<double> vel;
    bool cancel = false;
  };
  std::unordered_map<int64_t, Req> reqs;
  std::deque<int64_t> queue;
  int64_t next_id = 1;
  std::thread worker;
};

namespace {

double now_s(const lbm_server *s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

size_t nodes_of(const lbm_lattice_desc &d) {
  return (size_t)d.nx * d.ny * (d.lattice == LBM_D2Q9 ? 1 : d.nz);
}

// device bytes a running request allocates after its creation: the two FP64
// velocity snapshots of the residual (allocated by the first batch round)
// and, with keep_velocity, the FP64 staging of the final velocity query
size_t run_bytes(const lbm_request &r) {
  const size_t dn = nodes_of(r.lattice) * (r.lattice.lattice == LBM_D2Q9 ? 2 : 3);
  return (2 + (r.keep_velocity ? 1 : 0)) * dn * sizeof(double);
}

// device bytes of a request before it is created: two distribution arrays,
// flags and solid ids, the IBM fields, plus 10% and 1 MiB for the rest, and
// what it allocates while it runs
size_t estimate_bytes(const lbm_request &r) {
  const lbm_lattice_desc &d = r.lattice;
  const size_t n = nodes_of(d);
  const size_t q = d.lattice == LBM_D2Q9 ? 9 : 19;
  const size_t ssz = d.precision == LBM_FP64 ? 8 : d.precision == LBM_FP32 ? 4 : 2;
  const size_t tsz = d.precision == LBM_FP64 ? 8 : 4;
  size_t b = 2 * q * n * ssz + 3 * n;
  if (r.scheme.scheme == LBM_IBM_DIRECT) b += 6 * n * tsz;
  return b + b / 10 + (1u << 20) + run_bytes(r);
}

bool request_ok(const lbm_request &r) {
  const lbm_lattice_desc &d = r.lattice;
  if (d.lattice != LBM_D2Q9 && d.lattice != LBM_D3Q19) return false;
  if (d.nx < 1 || d.ny < 1 || (d.lattice == LBM_D3Q19 && d.nz < 1)) return false;
  if (!(d.tau > 0.5) || d.precision < LBM_FP64 || d.precision > LBM_FP32_FP16STORE) return false;
  if (r.nsolids < 0 || r.nsolids > 8) return false;
  if (r.scheme.scheme < LBM_SCHEME_NONE || r.scheme.scheme > LBM_ZHAO_YONG) return false;
  for (int k = 0; k < r.nsolids; k++)
    if (!(r.solids[k].radius > 0)) return false;
  return true;
}

lbm_status create_ctx(const lbm_request &r, cudaStream_t st, lbm_ctx **out) {
  *out = nullptr;
  lbm_ctx *c = nullptr;
  lbm_status s = lbm_create(&c, &r.lattice, st);
  if (s != LBM_OK) return s;
  for (int k = 0; k < r.nsolids && s == LBM_OK; k++) {
    int id = 0;
    s = lbm_add_solid(c, &r.solids[k], &id);
  }
  if (s == LBM_OK) s = lbm_set_scheme(c, &r.scheme);
  if (s == LBM_OK) s = lbm_init_equilibrium(c, r.rho0 > 0 ? r.rho0 : 1.0, r.u0);
  if (s != LBM_OK) {
    lbm_destroy(c);
    return s;
  }
  *out = c;
  return LBM_OK;
}

struct Active {
  int64_t id;
  lbm_ctx *ctx;
  size_t bytes;
  int64_t steps;
  bool retire;
};

void finish(lbm_server *s, Active &a, double residual, int status, int error) {
  lbm_result res;
  memset(&res, 0, sizeof(res));
  std::vector<double> vel;
  bool keep = false;
  int nsolids = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const lbm_request &r = s->reqs[a.id].r;
    keep = r.keep_velocity != 0;
    nsolids = r.nsolids;
  }
  const bool has_result = status == LBM_REQ_DONE || status == LBM_REQ_UNCONVERGED;
  if (a.ctx && has_result) {
    if (nsolids > 0) lbm_get_force_torque(a.ctx, 0, res.force, res.torque);
    if (keep) {
      lbm_info info;
      lbm_get_info(a.ctx, &info);
      lbm_lattice_desc d;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        d = s->reqs[a.id].r.lattice;
      }
      const size_t n = (size_t)info.nodes * (d.lattice == LBM_D2Q9 ? 2 : 3);
      vel.resize(n);
      if (lbm_get_velocity(a.ctx, vel.data(), n) != LBM_OK) vel.clear();
    }
  }
  // what the lattice held at the end, if that is above what admission
  // counted for it (it should not be)
  int64_t held = (int64_t)a.bytes;
  if (a.ctx) {
    lbm_info info;
    if (lbm_get_info(a.ctx, &info) == LBM_OK && info.device_bytes > held) held = info.device_bytes;
    lbm_destroy(a.ctx);
  }
  a.ctx = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  lbm_server::Req &q = s->reqs[a.id];
  q.res.device_bytes = held;
  q.res.status = status;
  q.res.error = error;
  q.res.steps = a.steps;
  q.res.residual = residual;
  for (int k = 0; k < 3; k++) {
    q.res.force[k] = res.force[k];
    q.res.torque[k] = res.torque[k];
  }
  q.res.finish_s = now_s(s);
  q.vel.swap(vel);
  s->cv_done.notify_all();
}

void fail_request(lbm_server *s, int64_t id, int error) {
  std::lock_guard<std::mutex> lk(s->mu);
  lbm_server::Req &q = s->reqs[id];
  q.res.status = LBM_REQ_FAILED;
  q.res.error = error;
  q.res.finish_s = now_s(s);
  s->cv_done.notify_all();
}

void run(lbm_server *s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
  std::vector<Active> act;
  lbm_batch *batch = nullptr;
  size_t used = 0;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (act.empty()) s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
      if (s->stop) break;
    }
    // admission, in submission order, by footprint
    bool changed = false;
    for (;;) {
      int64_t id;
      lbm_request r;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->queue.empty()) break;
        id = s->queue.front();
        r = s->reqs[id].r;
        if (r.deadline_s > 0 && now_s(s) > s->reqs[id].res.submit_s + r.deadline_s) {
          // expired while queued
          s->queue.pop_front();
          s->reqs[id].res.status = LBM_REQ_FAILED;
          s->reqs[id].res.error = LBM_ERR_TIMEOUT;
          s->reqs[id].res.finish_s = now_s(s);
          s->cv_done.notify_all();
          continue;
        }
        if (!act.empty() && used + estimate_bytes(r) > s->budget) break;
        s->queue.pop_front();
        s->reqs[id].res.status = LBM_REQ_RUNNING;
        s->reqs[id].res.start_s = now_s(s);
      }
      lbm_ctx *c = nullptr;
      const lbm_status cs = create_ctx(r, st, &c);
      if (cs != LBM_OK) {
        fail_request(s, id, cs);
        continue;
      }
      lbm_info info;
      lbm_get_info(c, &info);
      // its memory now plus what the batch rounds and the final query add
      const size_t bytes = (size_t)info.device_bytes + run_bytes(r);
      act.push_back({id, c, bytes, 0, false});
      used += bytes;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->reqs[id].res.device_bytes = (int64_t)bytes;
      }
      changed = true;
    }
    if (act.empty()) continue;
    if (changed && batch) {
      lbm_batch_destroy(batch);
      batch = nullptr;
    }
    lbm_status bs = LBM_OK;
    if (!batch) {
      std::vector<lbm_ctx *> ctxs;
      for (auto &a : act) ctxs.push_back(a.ctx);
      bs = lbm_batch_create(&batch, ctxs.data(), (int)ctxs.size(), st, 0);
    }
    std::vector<int64_t> steps(act.size(), 0);
    std::vector<double> res(act.size(), NAN);
    if (bs == LBM_OK)
      bs = lbm_batch_run_to_steady(batch, s->tol, s->check_every, s->check_every, steps.data(),
                                   res.data());
    // a member whose residual is not finite makes the round return
    // LBM_ERR_DIVERGED after the others have run their steps: only that
    // member fails, below.  Any other error fails the whole round.
    if (bs != LBM_OK && bs != LBM_ERR_DIVERGED) {
      if (batch) lbm_batch_destroy(batch);
      batch = nullptr;
      for (auto &a : act) {
        used -= a.bytes;
        finish(s, a, NAN, LBM_REQ_FAILED, bs);
      }
      act.clear();
      continue;
    }
    bool any = false;
    std::vector<int> why(act.size(), LBM_REQ_DONE);
    std::vector<int> err(act.size(), LBM_OK);
    for (size_t i = 0; i < act.size(); i++) {
      Active &a = act[i];
      a.steps += steps[i];
      if (!std::isfinite(res[i])) {
        a.retire = true;
        any = true;
        why[i] = LBM_REQ_FAILED;
        err[i] = LBM_ERR_DIVERGED;
        continue;
      }
      if (res[i] < s->tol) {
        a.retire = true;
        any = true;
      } else if (a.steps >= s->max_steps) {
        a.retire = true;
        any = true;
        why[i] = LBM_REQ_UNCONVERGED;
      }
      std::lock_guard<std::mutex> lk(s->mu);
      const lbm_server::Req &q = s->reqs[a.id];
      if (q.cancel) {
        a.retire = true;
        any = true;
        why[i] = LBM_REQ_CANCELLED;
      } else if (!(res[i] < s->tol) && q.r.deadline_s > 0 &&
                 now_s(s) > q.res.submit_s + q.r.deadline_s) {
        a.retire = true;
        any = true;
        why[i] = LBM_REQ_FAILED;
        err[i] = LBM_ERR_TIMEOUT;
      }
    }
    if (any) {
      // the batch gives the contexts their streams back before they go
      lbm_batch_destroy(batch);
      batch = nullptr;
      std::vector<Active> keep;
      for (size_t i = 0; i < act.size(); i++) {
        if (act[i].retire) {
          used -= act[i].bytes;
          finish(s, act[i], res[i], why[i], err[i]);
        } else {
          keep.push_back(act[i]);
        }
      }
      act.swap(keep);
    }
  }
  if (batch) lbm_batch_destroy(batch);
  for (auto &a : act) finish(s, a, NAN, LBM_REQ_FAILED, LBM_ERR_STATE);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (int64_t id : s->queue) {
      s->reqs[id].res.status = LBM_REQ_FAILED;
      s->reqs[id].res.error = LBM_ERR_STATE;
    }
    s->queue.clear();
    s->cv_done.notify_all();
  }
  if (st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
}

}  // namespace

extern "C" {

lbm_status lbm_server_create(lbm_server **out, size_t hbm_budget, double tol, int check_every,
                             int max_steps) {
  if (!out || hbm_budget == 0 || !(tol > 0) || check_every < 1 || max_steps < 1)
    return LBM_ERR_ARG;
  *out = nullptr;
  lbm_server *s = new lbm_server();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return LBM_ERR_CUDA;
  }
  s->budget = hbm_budget;
  s->tol = tol;
  s->check_every = check_every;
  s->max_steps = max_steps;
  s->t0 = std::chrono::steady_clock::now();
  s->worker = std::thread(run, s);
  *out = s;
  return LBM_OK;
}

lbm_status lbm_server_submit(lbm_server *s, const lbm_request *req, int64_t *id) {
  if (!s || !req || !id) return LBM_ERR_ARG;
  if (!request_ok(*req)) return LBM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return LBM_ERR_STATE;
  const int64_t k = s->next_id++;
  lbm_server::Req &q = s->reqs[k];
  q.r = *req;
  memset(&q.res, 0, sizeof(q.res));
  q.res.status = LBM_REQ_PENDING;
  q.res.residual = NAN;
  q.res.submit_s = now_s(s);
  s->queue.push_back(k);
  s->cv_work.notify_all();
  *id = k;
  return LBM_OK;
}

lbm_status lbm_server_poll(lbm_server *s, int64_t id, lbm_result *result) {
  if (!s || !result) return LBM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return LBM_ERR_ARG;
  *result = it->second.res;
  return LBM_OK;
}

lbm_status lbm_server_wait(lbm_server *s, int64_t id, lbm_result *result, double timeout_s) {
  if (!s || !result) return LBM_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return LBM_ERR_ARG;
  auto done = [&] {
    const int st = s->reqs[id].res.status;
    return st == LBM_REQ_DONE || st == LBM_REQ_FAILED || st == LBM_REQ_CANCELLED ||
           st == LBM_REQ_UNCONVERGED;
  };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
    *result = s->reqs[id].res;
    return LBM_ERR_TIMEOUT;
  }
  *result = s->reqs[id].res;
  return LBM_OK;
}

lbm_status lbm_server_velocity(lbm_server *s, int64_t id, double *host_out, size_t n) {
  if (!s || !host_out) return LBM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return LBM_ERR_ARG;
  const lbm_server::Req &q = it->second;
  if ((q.res.status != LBM_REQ_DONE && q.res.status != LBM_REQ_UNCONVERGED) || q.vel.empty())
    return LBM_ERR_STATE;
  if (n < q.vel.size()) return LBM_ERR_ARG;
  memcpy(host_out, q.vel.data(), q.vel.size() * sizeof(double));
  return LBM_OK;
}

lbm_status lbm_server_cancel(lbm_server *s, int64_t id) {
  if (!s) return LBM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return LBM_ERR_ARG;
  lbm_server::Req &q = it->second;
  if (q.res.status == LBM_REQ_PENDING) {
    for (auto qi = s->queue.begin(); qi != s->queue.end(); ++qi)
      if (*qi == id) {
        s->queue.erase(qi);
        break;
      }
    q.res.status = LBM_REQ_CANCELLED;
    q.res.finish_s = now_s(s);
    s->cv_done.notify_all();
    return LBM_OK;
  }
  if (q.res.status != LBM_REQ_RUNNING) return LBM_ERR_STATE;
  q.cancel = true;  // retired at the end of the round
  return LBM_OK;
}

void lbm_server_destroy(lbm_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  delete s;
}

}  // extern "C"
