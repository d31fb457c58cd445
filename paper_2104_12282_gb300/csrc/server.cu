// Request loop for gradient and optimisation requests on design domains of different sizes.
//
// The paper optimises one design at a time; serving many designs at once needs a runtime
// around the exact-gradient path.  This one is built on the public C ABI only:
//  * W worker threads, each with its own CUDA stream, take requests as soon as they are
//    free (continuous batching: a request that arrives while others run starts as soon as a
//    worker and memory are free, and its kernels overlap theirs on the GPU);
//  * grids stay resident on the device between requests of the same session (density,
//    displacement and multigrid state), and are evicted least-recently-used when memory
//    is needed;
//  * admission is by device memory: a request is started only when its grid is resident
//    or its estimated footprint fits the budget after evicting idle grids;
//  * the queue is served in arrival order among the requests that can be admitted.
// Each request's work runs in order on one stream and touches only its own grid, so its
// result is the one it gives alone.  With lockstep batching on (tomo_server_set_batching),
// a free worker takes the queued admissible gradient requests together and runs them as one
// tomo_batch: one CG loop for all of them, each phase one launch for every grid; results
// then agree with the request alone to the solver's tolerance.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/tomo.h"
#include "admission.h"
#include "host.h"

namespace {

using tomo_serve::Clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  int64_t ticket = 0;
  int64_t session = -1;
  tomo_grid_desc desc{};
  std::vector<uint8_t> fixed;
  std::vector<double> f;
  std::vector<float> z;
  float* dcdz = nullptr;  // caller-owned host outputs
  float* dvdz = nullptr;
  // optimisation request (iters > 0): OC iterations from z, final design into z_out
  int iters = 0;
  double volfrac = 0.0, move = 0.0;
  float* z_out = nullptr;
  size_t est_bytes = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  tomo_result res{};
  Clock::time_point t_submit, t_start, t_done;
};

}  // namespace

struct tomo_server {
  std::vector<std::thread> threads;
  std::vector<cudaStream_t> streams;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  int64_t next_ticket = 1;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  tomo_serve::Admission pool;  // resident grids, budget and eviction (under mu)
  tomo_server_stats stats{};
  std::string err;
  // lockstep batching: a free worker takes up to max_batch queued admissible gradient
  // requests at once and runs them as one tomo_batch (batch_workers streams); 1 = off
  int max_batch = 1;
  int batch_workers = 4;
  int64_t batches_run = 0;   // tomo_batch calls made for groups of two or more requests

  // An optimisation request on grid g (stream st): the design stays on the device for the
  // whole run (gradient with warm-started solves, then the OC update, iters times); the
  // compliance and solve info of the last gradient go to the result, the final design to
  // r.z_out.  The grid's warm-start setting is restored (off) afterwards.
  tomo_status optimise(tomo_grid* g, cudaStream_t st, Request& r) {
    const size_t ne = r.z.size();
    float* buf = nullptr;
    if (cudaMallocAsync((void**)&buf, sizeof(float) * 4 * ne, st) != cudaSuccess) {
      cudaGetLastError();
      return TOMO_ENOMEM;
    }
    float *z = buf, *zn = buf + ne, *dc = buf + 2 * ne, *dv = buf + 3 * ne;
    tomo_status s = TOMO_OK;
    if (cudaMemcpyAsync(z, r.z.data(), sizeof(float) * ne, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      s = TOMO_ECUDA;
    if (s == TOMO_OK) s = tomo_set_warm_start(g, 1);
    for (int k = 0; k < r.iters && s == TOMO_OK; ++k) {
      s = tomo_gradient(g, z, &r.res.compliance, dc, dv, &r.res.info);
      double change = 0.0;
      if (s == TOMO_OK) s = tomo_oc_step(g, z, dc, dv, r.volfrac, r.move, zn, &change);
      std::swap(z, zn);
    }
    tomo_set_warm_start(g, 0);
    if (s == TOMO_OK &&
        cudaMemcpyAsync(r.z_out, z, sizeof(float) * ne, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
      s = TOMO_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess && s == TOMO_OK) s = TOMO_ECUDA;
    cudaFreeAsync(buf, st);
    cudaGetLastError();
    return s;
  }

  // Fills r's message from m (truncated to the result's buffer).
  static void note(Request* r, const char* m) {
    const size_t n = std::min<size_t>(std::strlen(m), sizeof(r->res.message) - 1);
    std::memcpy(r->res.message, m, n);
    r->res.message[n] = 0;
    r->res.message_len = (int32_t)n;
  }

  // The grid of an admitted request's slot on stream st, created when the slot has none.
  tomo_status grid_for(Request* r, tomo_serve::Slot* slot, cudaStream_t st, tomo_grid** out) {
    tomo_grid* g = slot->grid;
    tomo_status s = TOMO_OK;
    if (!g) {
      tomo_grid_desc d = r->desc;
      d.fixed_dof = r->fixed.data();
      d.f = r->f.data();
      d.stream = st;
      s = tomo_create_grid(&d, &g);
      if (s != TOMO_OK) note(r, tomo_last_error(nullptr));
      std::lock_guard<std::mutex> lk(mu);
      slot->grid = g;
      if (s == TOMO_OK) stats.grids_created += 1;
    } else {
      tomo_set_stream(g, st);
    }
    *out = g;
    return s;
  }

  // One request alone on stream st (its grid already made).
  tomo_status run_one(Request* r, tomo_grid* g, cudaStream_t st) {
    nvtxRangePushA(r->iters > 0 ? "tomo server: optimisation request"
                                : "tomo server: gradient request");
    if (tomo::fault_hit(tomo::FAULT_SLOW))  // injected: a slow request (host wait)
      std::this_thread::sleep_for(std::chrono::milliseconds(200));
    tomo_status s;
    if (r->iters > 0) {
      s = optimise(g, st, *r);
    } else {
      s = tomo_gradient(g, r->z.data(), &r->res.compliance, r->dcdz, r->dvdz, &r->res.info);
      if (s == TOMO_OK && cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        s = TOMO_ECUDA;
      }
    }
    if (s != TOMO_OK) note(r, tomo_last_error(g));
    nvtxRangePop();
    return s;
  }

  // Gradient requests rs (grids gs) as one lockstep batch; on a batch failure each one is
  // run alone, so that one bad request does not fail the others.
  void run_group(std::vector<Request*>& rs, std::vector<tomo_grid*>& gs,
                 std::vector<tomo_status>& sts, cudaStream_t st) {
    const int n = (int)rs.size();
    tomo_batch* b = nullptr;
    tomo_status s = tomo_batch_create(batch_workers, &b);
    for (int i = 0; i < n && s == TOMO_OK; ++i) s = tomo_batch_append(b, gs[i]);
    if (s == TOMO_OK) {
      std::vector<const float*> z(n);
      std::vector<float*> dc(n), dv(n);
      std::vector<double> c(n);
      std::vector<tomo_solve_info> info(n);
      for (int i = 0; i < n; ++i) {
        z[i] = rs[i]->z.data();
        dc[i] = rs[i]->dcdz;
        dv[i] = rs[i]->dvdz;
      }
      s = tomo_batch_gradient(b, z.data(), c.data(), dc.data(), dv.data(), info.data());
      if (s == TOMO_OK) {
        for (int i = 0; i < n; ++i) {
          rs[i]->res.compliance = c[i];
          rs[i]->res.info = info[i];
          sts[i] = TOMO_OK;
        }
        std::lock_guard<std::mutex> lk(mu);
        batches_run += 1;
      }
    }
    if (b) tomo_batch_destroy(b);
    for (int i = 0; i < n; ++i) tomo_set_stream(gs[i], st);
    if (s != TOMO_OK)
      for (int i = 0; i < n; ++i) sts[i] = run_one(rs[i], gs[i], st);
  }

  void work(int w) {
    cudaStream_t st = streams[w];
    for (;;) {
      std::vector<Request*> rs;
      std::vector<tomo_serve::Slot*> slots;
      std::vector<tomo_grid*> dead;
      {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
          if (stop) return;
          // the first admissible request in arrival order, then (batching) the further
          // admissible gradient requests behind it, up to max_batch
          for (size_t k = 0; k < queue.size();) {
            Request& q = *reqs[queue[k]];
            const bool joins = rs.empty() || (max_batch > 1 && q.iters == 0 &&
                                              rs[0]->iters == 0 && (int)rs.size() < max_batch);
            tomo_serve::Slot* slot = joins ? pool.admit(q.session, q.desc, q.est_bytes, dead)
                                           : nullptr;
            if (slot) {
              rs.push_back(&q);
              slots.push_back(slot);
              queue.erase(queue.begin() + k);
              if (q.iters > 0 || max_batch <= 1) break;
            } else {
              ++k;
            }
          }
          if (!rs.empty()) break;
          cv_work.wait(lk);
        }
        for (Request* r : rs) {
          r->state = 1;
          r->t_start = Clock::now();
        }
        stats.evictions = pool.evictions;
        stats.peak_bytes = std::max<uint64_t>(stats.peak_bytes, pool.resident);
      }
      for (tomo_grid* e : dead) {  // evicted idle grids: quiesce on this worker's stream
        tomo_set_stream(e, st);
        tomo_destroy_grid(e);
      }
      dead.clear();
      // the slots are busy: this worker alone touches their grids until released below
      const int n = (int)rs.size();
      std::vector<tomo_grid*> gs(n, nullptr);
      std::vector<tomo_status> sts(n, TOMO_OK);
      std::vector<Request*> grs;
      std::vector<tomo_grid*> ggs;
      std::vector<int> gi;
      for (int i = 0; i < n; ++i) {
        sts[i] = grid_for(rs[i], slots[i], st, &gs[i]);
        if (sts[i] != TOMO_OK) continue;
        if (n == 1) {
          sts[i] = run_one(rs[i], gs[i], st);
        } else {
          grs.push_back(rs[i]);
          ggs.push_back(gs[i]);
          gi.push_back(i);
        }
      }
      if (!grs.empty()) {
        std::vector<tomo_status> gst(grs.size(), TOMO_OK);
        if (grs.size() == 1) gst[0] = run_one(grs[0], ggs[0], st);
        else run_group(grs, ggs, gst, st);
        for (size_t k = 0; k < gi.size(); ++k) sts[gi[k]] = gst[k];
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        const auto t = Clock::now();
        for (int i = 0; i < n; ++i) {
          Request* r = rs[i];
          r->t_done = t;
          r->res.status = sts[i];
          r->res.queue_ms = ms_between(r->t_submit, r->t_start);
          r->res.run_ms = ms_between(r->t_start, r->t_done);
          r->state = 2;
          stats.completed += 1;
          // no session (or a failure): the grid is freed at once
          pool.release(slots[i], sts[i] == TOMO_OK && r->session >= 0, r->t_done, dead);
        }
      }
      for (tomo_grid* e : dead) {
        tomo_set_stream(e, st);
        tomo_destroy_grid(e);
      }
      dead.clear();
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

namespace {

tomo_status submit_request(tomo_server* S, const tomo_grid_desc* desc, int64_t session,
                           const float* z, float* dcdz, float* dvdz, int iters, double volfrac,
                           double move, float* z_out, int64_t* ticket) {
  if (desc->precision != TOMO_FP32) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->err = "the request loop serves FP32 grids";
    return TOMO_EINVAL;
  }
  if (desc->nx < 1 || desc->ny < 1 || desc->nz < 1) return TOMO_EINVAL;
  auto r = std::make_unique<Request>();
  r->session = session;
  r->desc = *desc;
  const size_t nn = (size_t)(desc->nx + 1) * (desc->ny + 1) * (desc->nz + 1);
  const size_t ne = (size_t)desc->nx * desc->ny * desc->nz;
  r->fixed.assign(desc->fixed_dof, desc->fixed_dof + 3 * nn);
  r->f.assign(desc->f, desc->f + 3 * nn);
  r->z.assign(z, z + ne);
  r->desc.fixed_dof = nullptr;
  r->desc.f = nullptr;
  r->desc.stream = nullptr;
  r->dcdz = dcdz;
  r->dvdz = dvdz;
  r->iters = iters;
  r->volfrac = volfrac;
  r->move = move;
  r->z_out = z_out;
  size_t est = 0;
  tomo_estimate_device_bytes(desc, &est);
  if (iters > 0) est += sizeof(float) * 4 * ne;  // the run's design and gradient buffers
  r->est_bytes = est;
  std::lock_guard<std::mutex> lk(S->mu);
  if (est > S->pool.budget) {
    S->err = "request needs more device memory than the server's budget";
    return TOMO_ENOMEM;
  }
  r->t_submit = Clock::now();
  r->ticket = S->next_ticket++;
  *ticket = r->ticket;
  S->queue.push_back(r->ticket);
  S->reqs[r->ticket] = std::move(r);
  S->stats.submitted += 1;
  S->cv_work.notify_one();
  return TOMO_OK;
}

}  // namespace

extern "C" {

tomo_status tomo_server_create(int32_t workers, uint64_t budget_bytes, tomo_server** out) {
  if (!out || budget_bytes == 0) return TOMO_EINVAL;
  *out = nullptr;
  if (workers <= 0) workers = 8;
  if (workers > 64) workers = 64;
  std::unique_ptr<tomo_server> S(new (std::nothrow) tomo_server());
  if (!S) return TOMO_ENOMEM;
  S->pool.budget = (size_t)budget_bytes;
  for (int w = 0; w < workers; ++w) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (auto t : S->streams) cudaStreamDestroy(t);
      return TOMO_ECUDA;
    }
    S->streams.push_back(s);
  }
  int dev = 0;
  cudaGetDevice(&dev);
  for (int w = 0; w < workers; ++w)
    S->threads.emplace_back([srv = S.get(), w, dev] {
      cudaSetDevice(dev);
      srv->work(w);
    });
  *out = S.release();
  return TOMO_OK;
}


tomo_status tomo_server_submit(tomo_server* S, const tomo_grid_desc* desc, int64_t session,
                               const float* z, float* dcdz, float* dvdz, int64_t* ticket) {
  if (!S || !desc || !z || !dcdz || !ticket || !desc->fixed_dof || !desc->f) return TOMO_EINVAL;
  return submit_request(S, desc, session, z, dcdz, dvdz, 0, 0.0, 0.0, nullptr, ticket);
}

tomo_status tomo_server_submit_optimize(tomo_server* S, const tomo_grid_desc* desc,
                                        int64_t session, const float* z, int32_t iters,
                                        double volfrac, double move, float* z_out,
                                        int64_t* ticket) {
  if (!S || !desc || !z || !z_out || !ticket || !desc->fixed_dof || !desc->f || iters < 1 ||
      !(volfrac > 0.0 && volfrac <= 1.0) || !(move > 0.0))
    return TOMO_EINVAL;
  return submit_request(S, desc, session, z, nullptr, nullptr, iters, volfrac, move, z_out,
                        ticket);
}

tomo_status tomo_server_wait(tomo_server* S, int64_t ticket, tomo_result* result) {
  if (!S || !result) return TOMO_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    S->err = "unknown ticket";
    return TOMO_EINVAL;
  }
  S->cv_done.wait(lk, [&] { return it->second->state == 2; });
  *result = it->second->res;
  result->ticket = ticket;
  S->reqs.erase(it);
  return TOMO_OK;
}

tomo_status tomo_server_get_stats(tomo_server* S, tomo_server_stats* st) {
  if (!S || !st) return TOMO_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  *st = S->stats;
  st->evictions = S->pool.evictions;
  st->resident_bytes = S->pool.resident;
  st->resident_grids = (int32_t)S->pool.slots.size();
  st->queued = (int32_t)S->queue.size();
  st->batches = S->batches_run;
  return TOMO_OK;
}

tomo_status tomo_server_set_batching(tomo_server* S, int32_t max_batch, int32_t batch_workers) {
  if (!S) return TOMO_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  S->max_batch = std::max<int32_t>(1, std::min<int32_t>(max_batch, 256));
  S->batch_workers = batch_workers > 0 ? std::min<int32_t>(batch_workers, 64) : 4;
  return TOMO_OK;
}

tomo_status tomo_server_destroy(tomo_server* S) {
  if (!S) return TOMO_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->threads) t.join();
  for (auto& s : S->pool.slots)
    if (s->grid) tomo_destroy_grid(s->grid);
  for (auto s : S->streams) cudaStreamDestroy(s);
  delete S;
  return TOMO_OK;
}

const char* tomo_server_last_error(const tomo_server* S) {
  if (!S) return "";
  // a copy per calling thread: another thread's submit may replace the message meanwhile
  static thread_local std::string copy;
  std::lock_guard<std::mutex> lk(const_cast<tomo_server*>(S)->mu);
  copy = S->err;
  return copy.c_str();
}

}  // extern "C"
