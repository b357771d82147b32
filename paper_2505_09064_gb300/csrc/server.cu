// Request server (include/vasmg.h, "serving"): continuous admission of
// independent problems onto one device.  Host code only; every request runs
// through the public entry points (vasmg_setup, vasmg_solve_multi,
// vasmg_destroy), so its result is the one those calls give alone.
//
// Worker threads ("slots") each own a non-blocking stream.  A free slot takes
// the head of the arrival queue once the head's estimated device footprint
// fits the unused part of the memory budget (the head runs alone if it can
// never fit).  The slot sets up the request's hierarchy, keeps it resident
// while it solves all right-hand sides together (one multi solve), writes U,
// destroys the hierarchy and
// returns the footprint to the budget.  Slots run concurrently, so requests
// overlap on the device; each handle's sweep grids are capped to a share of
// the device (vasmg_options.max_ctas) so that all running sweeps can be
// resident together, which their cross-CTA waits require.
//
// Batched mode (vasmg_server_opts.batch): a slot sets up its request and hands
// the hierarchy to one executor thread, which repeatedly takes every request
// ready at that moment and solves one right-hand side of each with
// vasmg_solve_batch (one launch per level and phase for all of them); a
// request with more right-hand sides rejoins the next round.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/vasmg.h"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Owned copy of one request.
struct Request {
  uint64_t id = 0;
  int32_t dim = 2;
  int64_t nv = 0, ne = 0;
  std::vector<double> coords, lam, mu, dvals;
  std::vector<int32_t> elems;
  std::vector<int64_t> ddofs;
  double lam_c = 0, mu_c = 0;
  bool has_lam = false, has_mu = false, has_dvals = false;
  std::vector<std::vector<double>> F;
  std::vector<double*> U;
  int64_t footprint = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  vasmg_request_stats st{};
  bool done = false;
};

// Device bytes a request is expected to hold at its peak (setup sorts and the
// Galerkin products dominate): per vertex and per element, by dimension.
// The multi solve holds its right-hand sides in passes of 2, 4 or 8: about
// 80 bytes per dof and right-hand side of a pass (CG and V-cycle vectors).
int64_t footprint_estimate(int dim, int64_t nv, int64_t ne, int32_t nrhs) {
  const int64_t per_v = dim == 2 ? 4096 : 16384;
  const int64_t pass = nrhs <= 1 ? 1 : (nrhs <= 2 ? 2 : (nrhs <= 4 ? 4 : 8));
  return per_v * nv + 96 * ne + (16 * (int64_t)nrhs + 80 * pass) * nv * dim + (32ll << 20);
}

}  // namespace

struct vasmg_server {
  // a request's hierarchy waiting for, or in, a batched round
  struct Job {
    vasmg_handle h = nullptr;
    Request* r = nullptr;
    size_t next = 0;          // right-hand sides solved so far
    bool finished = false;
    int status = VASMG_OK;
  };
  vasmg_server_opts o{};
  int device = 0;
  int max_ctas = 0;
  int64_t budget = 0, used = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
  uint64_t next_id = 1;
  bool stop = false;
  std::vector<std::thread> workers;
  std::deque<Job*> ready;               // batched mode
  std::condition_variable cv_ready, cv_solved;
  bool stop_exec = false;
  std::thread executor;

  // Batched mode: one right-hand side of every ready request per round.
  void executor_loop() {
    cudaSetDevice(device);
    for (;;) {
      std::vector<Job*> batch;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_ready.wait(lk, [&] { return !ready.empty() || stop_exec; });
        if (ready.empty()) break;
        while (!ready.empty()) {
          batch.push_back(ready.front());
          ready.pop_front();
        }
      }
      const int32_t k = (int32_t)batch.size();
      std::vector<vasmg_handle> hs(k);
      std::vector<const double*> Fp(k);
      std::vector<double*> Up(k);
      std::vector<vasmg_stats> ss(k);
      for (int32_t i = 0; i < k; ++i) {
        hs[i] = batch[i]->h;
        Fp[i] = batch[i]->r->F[batch[i]->next].data();
        Up[i] = batch[i]->r->U[batch[i]->next];
      }
      const int rc = vasmg_solve_batch(k, hs.data(), Fp.data(), Up.data(), o.tol, ss.data());
      {
        std::lock_guard<std::mutex> lk(mu);
        for (int32_t i = 0; i < k; ++i) {
          Job* j = batch[i];
          vasmg_request_stats& st = j->r->st;
          if (rc < 0) {
            j->status = rc;
            j->finished = true;
            continue;
          }
          st.iterations += ss[i].iterations;
          st.max_iterations = std::max(st.max_iterations, ss[i].iterations);
          st.max_rel_res = std::max(st.max_rel_res, ss[i].rel_res);
          if (!(ss[i].rel_res < o.tol)) j->status = std::max(j->status, (int)VASMG_NOT_CONVERGED);
          if (++j->next == j->r->F.size()) j->finished = true;
          else ready.push_back(j);
        }
      }
      cv_solved.notify_all();
    }
  }

  void run(Request* r, cudaStream_t stream) {
    vasmg_problem pb{};
    pb.dim = r->dim;
    pb.n_vertices = r->nv;
    pb.coords = r->coords.data();
    pb.n_elements = r->ne;
    pb.elements = r->elems.data();
    pb.lambda = r->has_lam ? r->lam.data() : nullptr;
    pb.mu = r->has_mu ? r->mu.data() : nullptr;
    pb.lambda_const = r->lam_c;
    pb.mu_const = r->mu_c;
    pb.n_dirichlet = (int64_t)r->ddofs.size();
    pb.dirichlet_dofs = r->ddofs.empty() ? nullptr : r->ddofs.data();
    pb.dirichlet_values = r->has_dvals ? r->dvals.data() : nullptr;
    vasmg_options opt;
    vasmg_default_options(r->dim, &opt);
    opt.precision = o.precision;
    opt.max_iters = o.max_iters;
    opt.max_ctas = max_ctas;
    // lanes per row by rule: a request's latency carries no tuning runs
    opt.autotune = 0;
    opt.stream = stream;
    vasmg_request_stats& st = r->st;
    st.n_rhs = (int32_t)r->F.size();
    vasmg_handle h = nullptr;
    const double t0 = now_ms();
    int rc = vasmg_setup(&pb, &opt, &h);
    st.setup_ms = now_ms() - t0;
    int worst = rc;
    if (rc == VASMG_OK && o.batch) {
      const double t1 = now_ms();
      Job j;
      j.h = h;
      j.r = r;
      {
        std::unique_lock<std::mutex> lk(mu);
        ready.push_back(&j);
        cv_ready.notify_all();
        cv_solved.wait(lk, [&] { return j.finished; });
      }
      worst = j.status;
      st.solve_ms = now_ms() - t1;
    } else if (rc == VASMG_OK) {
      // every right-hand side of the request in one multi solve: each sweep
      // reads the hierarchy once for all of them, and each result is the one
      // vasmg_solve gives alone
      const double t1 = now_ms();
      const int32_t k = (int32_t)r->F.size();
      std::vector<const double*> Fp(k);
      for (int32_t i = 0; i < k; ++i) Fp[i] = r->F[i].data();
      std::vector<vasmg_stats> ss(k);
      rc = vasmg_solve_multi(h, k, Fp.data(), r->U.data(), o.tol, ss.data());
      worst = rc;
      if (rc >= 0)
        for (int32_t i = 0; i < k; ++i) {
          st.iterations += ss[i].iterations;
          st.max_iterations = std::max(st.max_iterations, ss[i].iterations);
          st.max_rel_res = std::max(st.max_rel_res, ss[i].rel_res);
        }
      st.solve_ms = now_ms() - t1;
    }
    if (h) vasmg_destroy(h);
    st.status = worst;
  }

  void worker() {
    cudaSetDevice(device);
    cudaStream_t stream = nullptr;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) stream = nullptr;
    for (;;) {
      Request* r = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] {
          if (queue.empty()) return stop;
          const int64_t fp = queue.front()->footprint;
          return used + fp <= budget || used == 0;
        });
        if (queue.empty()) break;  // stop requested and nothing left
        r = queue.front();
        queue.pop_front();
        used += r->footprint;
        r->t_admit = now_ms();
      }
      cv_work.notify_all();
      run(r, stream);
      {
        std::lock_guard<std::mutex> lk(mu);
        used -= r->footprint;
        r->t_done = now_ms();
        r->st.queue_ms = r->t_admit - r->t_submit;
        r->st.latency_ms = r->t_done - r->t_submit;
        r->st.footprint_bytes = r->footprint;
        r->done = true;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
    if (stream) {
      cudaStreamSynchronize(stream);
      cudaStreamDestroy(stream);
    }
  }
};

extern "C" {

int vasmg_server_default_opts(vasmg_server_opts* out) {
  if (!out) return VASMG_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->slots = 4;
  out->precision = VASMG_FP32_VCYCLE;
  out->max_iters = 1000;
  out->tol = 1e-6;
  out->memory_budget = 0;
  out->batch = 0;
  return VASMG_OK;
}

int vasmg_server_create(const vasmg_server_opts* opts, vasmg_server** out) {
  if (!out) return VASMG_ERR_INVALID_ARG;
  *out = nullptr;
  vasmg_server_opts o;
  if (opts) o = *opts; else vasmg_server_default_opts(&o);
  if (o.slots <= 0 || o.slots > 64 || !(o.tol > 0.0) || o.max_iters <= 0 || o.memory_budget < 0 ||
      o.precision < VASMG_FP64 || o.precision > VASMG_FP32_VCYCLE_BF16_SMOOTH || o.batch < 0 || o.batch > 1)
    return VASMG_ERR_INVALID_ARG;
  try {
    std::unique_ptr<vasmg_server> s(new vasmg_server());
    s->o = o;
    if (cudaGetDevice(&s->device) != cudaSuccess) return VASMG_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) return VASMG_ERR_CUDA;
    // every sweep kernel holds at least two CTAs per SM
    s->max_ctas = std::max(1, 2 * sms / o.slots);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return VASMG_ERR_CUDA;
    s->budget = o.memory_budget > 0 ? o.memory_budget : (int64_t)(free_b / 2);
    if (o.batch) s->executor = std::thread([p = s.get()] { p->executor_loop(); });
    for (int i = 0; i < o.slots; ++i) s->workers.emplace_back([p = s.get()] { p->worker(); });
    *out = s.release();
    return VASMG_OK;
  } catch (const std::bad_alloc&) {
    return VASMG_ERR_OOM;
  } catch (...) {
    return VASMG_ERR_UNSUPPORTED;
  }
}

int vasmg_server_submit(vasmg_server* s, const vasmg_problem* pb, int32_t n_rhs, const double* const* F,
                        double* const* U, uint64_t* ticket) {
  if (!s || !pb || !F || !U || !ticket || n_rhs <= 0) return VASMG_ERR_INVALID_ARG;
  if ((pb->dim != 2 && pb->dim != 3) || pb->n_vertices <= 0 || pb->n_elements <= 0 || !pb->coords || !pb->elements ||
      pb->n_dirichlet < 0 || (pb->n_dirichlet > 0 && !pb->dirichlet_dofs))
    return VASMG_ERR_INVALID_ARG;
  for (int32_t i = 0; i < n_rhs; ++i)
    if (!F[i] || !U[i]) return VASMG_ERR_INVALID_ARG;
  try {
    std::unique_ptr<Request> r(new Request());
    const int d = pb->dim;
    r->dim = d;
    r->nv = pb->n_vertices;
    r->ne = pb->n_elements;
    r->coords.assign(pb->coords, pb->coords + r->nv * d);
    r->elems.assign(pb->elements, pb->elements + r->ne * (d + 1));
    if (pb->lambda) {
      r->has_lam = true;
      r->lam.assign(pb->lambda, pb->lambda + r->ne);
    }
    if (pb->mu) {
      r->has_mu = true;
      r->mu.assign(pb->mu, pb->mu + r->ne);
    }
    r->lam_c = pb->lambda_const;
    r->mu_c = pb->mu_const;
    if (pb->n_dirichlet > 0) r->ddofs.assign(pb->dirichlet_dofs, pb->dirichlet_dofs + pb->n_dirichlet);
    if (pb->dirichlet_values) {
      r->has_dvals = true;
      r->dvals.assign(pb->dirichlet_values, pb->dirichlet_values + pb->n_dirichlet);
    }
    const int64_t n = r->nv * d;
    r->F.resize(n_rhs);
    for (int32_t i = 0; i < n_rhs; ++i) r->F[i].assign(F[i], F[i] + n);
    r->U.assign(U, U + n_rhs);
    r->footprint = footprint_estimate(d, r->nv, r->ne, n_rhs);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->stop) return VASMG_ERR_INVALID_ARG;
      r->id = s->next_id++;
      r->t_submit = now_ms();
      *ticket = r->id;
      s->queue.push_back(r.get());
      s->all.emplace(r->id, std::move(r));
    }
    s->cv_work.notify_all();
    return VASMG_OK;
  } catch (const std::bad_alloc&) {
    return VASMG_ERR_OOM;
  }
}

int vasmg_server_poll(vasmg_server* s, uint64_t ticket, int32_t wait_ms, vasmg_request_stats* st) {
  if (!s) return VASMG_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return VASMG_ERR_INVALID_ARG;
  Request* r = it->second.get();
  auto done = [&] { return r->done; };
  if (wait_ms < 0)
    s->cv_done.wait(lk, done);
  else
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), done);
  if (!r->done) return VASMG_PENDING;
  if (st) *st = r->st;
  s->all.erase(it);
  return VASMG_OK;
}

int vasmg_server_destroy(vasmg_server* s) {
  if (!s) return VASMG_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  if (s->executor.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop_exec = true;
    }
    s->cv_ready.notify_all();
    s->executor.join();
  }
  delete s;
  return VASMG_OK;
}

}  // extern "C"
