// extern "C" entry points of libvasmg (declared in include/vasmg.h).  Every
// entry point catches internal exceptions and returns an error code.
#include <chrono>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace vasmg;

struct vasmg_ctx {
  Ctx c;
};

namespace {

thread_local std::string g_last_error;

int fail(const std::exception& e) {
  g_last_error = e.what();
  if (const Error* v = dynamic_cast<const Error*>(&e)) return v->code;
  return VASMG_ERR_CUDA;
}

#define VASMG_API_BEGIN try {
#define VASMG_API_END                           \
  }                                             \
  catch (const std::bad_alloc& e) {             \
    g_last_error = e.what();                    \
    return VASMG_ERR_OOM;                       \
  }                                             \
  catch (const std::exception& e) {             \
    return fail(e);                             \
  }

void destroy_ctx(vasmg_ctx* h) {
  cudaStream_t s = h->c.stream;
  cudaEvent_t ev = h->c.join_ev, nev = h->c.noalloc_ev;
  destroy_solver_state(h->c);
  delete h;
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  if (ev) cudaEventDestroy(ev);
  if (nev) {
    cudaEventSynchronize(nev);
    cudaEventDestroy(nev);
  }
}

// Scratch of vasmg_coarse_solve_noalloc: static device memory, so the call
// never allocates.  In host code the name is only a host-side stand-in; the
// device address is looked up with cudaGetSymbolAddress once per device and
// context (a context created after a reset loads the module again, and the
// array may then sit elsewhere) and passed to the kernel.
__device__ __align__(256) double g_noalloc_scratch[VASMG_NOALLOC_MAX_DOFS];
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoallocSlot {
  unsigned long long ctx_id = 0;  // 0: not looked up yet
  double* ptr = nullptr;
};
NoallocSlot g_noalloc_slot[kMaxDevices];

// cuCtxGetCurrent / cuCtxGetId through the runtime's driver entry points (the
// library links the runtime statically and not libcuda): the id of the current
// context, unique for the life of the process.  0 if unavailable.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = (CtxGetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)f;
    cudaGetLastError();
  });
  if (!get_cur || !get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Coarsest solve into x from b (canonical dof order): copy b into the scratch,
// substitute with the FP64 Cholesky factor (the same routine as the V-cycle's
// coarsest solve), copy out.  One warp.
__global__ void coarse_noalloc_kernel(const double* __restrict__ chol, const uint8_t* __restrict__ drop, int n,
                                      const double* b, double* x, double* y) {
  const int lane = threadIdx.x & 31;
  for (int t = lane; t < n; t += 32) y[t] = b[t];
  __syncwarp();
  chol_substitute_warp(chol, drop, n, y);
  for (int t = lane; t < n; t += 32) x[t] = y[t];
}

// True if p is device (or managed) memory on device dev.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

extern "C" {

int vasmg_default_options(int dim, vasmg_options* out) {
  if (!out || (dim != 2 && dim != 3)) return VASMG_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->leaf_threshold = dim == 2 ? 4 : 8;
  out->n_pre = 1;
  out->n_post = 1;
  out->precision = VASMG_FP64;
  out->coarse_max_dofs = 0;
  out->max_iters = 1000;
  out->use_graph = 1;
  out->dense_coarse = 1;
  out->autotune = 1;
  out->stream = nullptr;
  out->cycle = 1;
  out->additive = 0;
  return VASMG_OK;
}

int vasmg_setup(const vasmg_problem* pb, const vasmg_options* opt, vasmg_handle* out) {
  if (!pb || !out) return VASMG_ERR_INVALID_ARG;
  *out = nullptr;
  const int d = pb->dim;
  if ((d != 2 && d != 3) || pb->n_vertices <= 0 || pb->n_elements <= 0 || !pb->coords || !pb->elements)
    return VASMG_ERR_INVALID_ARG;
  if (pb->n_vertices >= (int64_t)INT32_MAX / 4 || pb->n_elements >= (int64_t)INT32_MAX / 4)
    return VASMG_ERR_UNSUPPORTED;
  if (pb->n_dirichlet < 0 || (pb->n_dirichlet > 0 && !pb->dirichlet_dofs)) return VASMG_ERR_INVALID_ARG;
  vasmg_options o;
  if (opt) o = *opt; else vasmg_default_options(d, &o);
  if (o.n_pre != 1 || o.n_post != 1) return VASMG_ERR_UNSUPPORTED;
  if (o.precision < VASMG_FP64 || o.precision > VASMG_FP32_VCYCLE_BF16_SMOOTH) return VASMG_ERR_INVALID_ARG;
  if (o.coarse_max_dofs < 0 || o.coarse_max_dofs > 4096 || o.max_iters <= 0 || o.max_ctas < 0 ||
      o.dense_coarse < 0 || o.dense_coarse > 1 || o.autotune < 0 || o.autotune > 1 || o.cycle < 0 ||
      o.cycle > 4 || o.additive < 0 || o.additive > 1)
    return VASMG_ERR_INVALID_ARG;
  vasmg_ctx* h = new vasmg_ctx();
  struct Guard {
    vasmg_ctx*& h;
    bool armed = true;
    ~Guard() {
      if (armed && h) destroy_ctx(h);
    }
  } guard{h};
  VASMG_API_BEGIN
  const double t0 = now_ms();
  Ctx& c = h->c;
  c.dim = d;
  c.K = d == 2 ? 31 : 20;
  c.T = o.leaf_threshold > 0 ? o.leaf_threshold : (d == 2 ? 4 : 8);
  c.precision = o.precision;
  c.max_iters = o.max_iters;
  c.use_graph = o.use_graph;
  c.max_ctas = o.max_ctas > 0 ? o.max_ctas : 0;
  c.dense_coarse = o.dense_coarse;
  c.autotune = o.autotune;
  c.gamma = o.cycle > 0 ? o.cycle : 1;
  c.additive = o.additive;
  c.coarse_max_dofs = o.coarse_max_dofs;
  c.user_stream = (cudaStream_t)o.stream;
  VASMG_CUDA(cudaGetDevice(&c.device));
  VASMG_CUDA(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
  VASMG_CUDA(cudaEventCreateWithFlags(&c.join_ev, cudaEventDisableTiming));
  VASMG_CUDA(cudaEventCreateWithFlags(&c.noalloc_ev, cudaEventDisableTiming));
  join_user(c);
  c.nv = pb->n_vertices;
  c.ne = pb->n_elements;
  c.n = c.nv * d;
  cudaStream_t s = c.stream;
  // inputs
  std::vector<uint8_t> isdir((size_t)c.n, 0);
  std::vector<double> udir((size_t)c.n, 0.0);
  c.dir_dofs.assign(pb->dirichlet_dofs, pb->dirichlet_dofs + pb->n_dirichlet);
  for (int64_t k = 0; k < pb->n_dirichlet; ++k) {
    const int64_t g = pb->dirichlet_dofs[k];
    VASMG_CHECK(g >= 0 && g < c.n, VASMG_ERR_INVALID_ARG, "Dirichlet dof out of range");
    isdir[g] = 1;
    udir[g] = pb->dirichlet_values ? pb->dirichlet_values[k] : 0.0;
    if (pb->dirichlet_values && pb->dirichlet_values[k] != 0.0) c.has_dir_values = true;
  }
  for (int64_t i = 0; i < c.n; ++i)
    VASMG_CHECK(std::isfinite(pb->coords[i]), VASMG_ERR_INVALID_ARG, "non-finite coordinate");
  c.X.alloc(c.n, s);
  c.X.upload(pb->coords, c.n);
  c.E.alloc(c.ne * (d + 1), s);
  c.E.upload(pb->elements, c.ne * (d + 1));
  std::vector<double> lam((size_t)c.ne), mu((size_t)c.ne);
  for (int64_t e = 0; e < c.ne; ++e) {
    lam[e] = pb->lambda ? pb->lambda[e] : pb->lambda_const;
    mu[e] = pb->mu ? pb->mu[e] : pb->mu_const;
  }
  c.lam.alloc(c.ne, s);
  c.lam.upload(lam.data(), c.ne);
  c.mu.alloc(c.ne, s);
  c.mu.upload(mu.data(), c.ne);
  c.isdir.alloc(c.n, s);
  c.isdir.upload(isdir.data(), c.n);
  c.udir.alloc(c.n, s);
  c.udir.upload(udir.data(), c.n);
  c.C.resize(1);
  setup_assemble(c);
  setup_tree(c);
  setup_colour_and_solve_levels(c);
  setup_solver_state(c);
  VASMG_CUDA(cudaStreamSynchronize(s));
  c.setup_ms = now_ms() - t0;
  *out = h;
  guard.armed = false;
  return VASMG_OK;
  VASMG_API_END
}

int vasmg_update_data(vasmg_handle h, const double* lambda, const double* mu, double lambda_const, double mu_const,
                      const double* dirichlet_values) {
  if (!h) return VASMG_ERR_INVALID_ARG;
  VASMG_API_BEGIN
  const double t0 = now_ms();
  Ctx& c = h->c;
  join_user(c);
  cudaStream_t s = c.stream;
  // a vasmg_coarse_solve_noalloc kernel still reading the factor finishes first
  VASMG_CUDA(cudaStreamWaitEvent(s, c.noalloc_ev, 0));
  std::vector<double> lam((size_t)c.ne), mu_v((size_t)c.ne);
  for (int64_t e = 0; e < c.ne; ++e) {
    lam[e] = lambda ? lambda[e] : lambda_const;
    mu_v[e] = mu ? mu[e] : mu_const;
    VASMG_CHECK(std::isfinite(lam[e]) && std::isfinite(mu_v[e]), VASMG_ERR_INVALID_ARG, "non-finite Lame parameter");
  }
  c.lam.upload(lam.data(), c.ne);
  c.mu.upload(mu_v.data(), c.ne);
  if (dirichlet_values) {
    std::vector<double> udir((size_t)c.n, 0.0);
    c.has_dir_values = false;
    for (size_t k = 0; k < c.dir_dofs.size(); ++k) {
      udir[(size_t)c.dir_dofs[k]] = dirichlet_values[k];
      if (dirichlet_values[k] != 0.0) c.has_dir_values = true;
    }
    c.udir.upload(udir.data(), c.n);
  }
  assemble_values(c);
  for (int l = 0; l + 1 < (int)c.C.size(); ++l) galerkin_values(c, l);
  solve_level_values(c);
  refresh_solver_values(c);
  VASMG_CUDA(cudaStreamSynchronize(s));
  c.update_ms = now_ms() - t0;
  return VASMG_OK;
  VASMG_API_END
}

int vasmg_assemble_load(vasmg_handle h, const double* body_force, double* F) {
  if (!h || !body_force || !F) return VASMG_ERR_INVALID_ARG;
  VASMG_API_BEGIN
  Ctx& c = h->c;
  join_user(c);
  DevBuf<double> tmp;
  tmp.alloc(c.n, c.stream);
  assemble_load_dev(c, body_force, tmp.get());
  VASMG_CUDA(cudaMemcpyAsync(F, tmp.get(), sizeof(double) * c.n, cudaMemcpyDefault, c.stream));
  VASMG_CUDA(cudaStreamSynchronize(c.stream));
  return VASMG_OK;
  VASMG_API_END
}

int vasmg_solve(vasmg_handle h, const double* F, double* U, double tol, vasmg_stats* st) {
  if (!h || !F || !U || !(tol > 0.0)) return VASMG_ERR_INVALID_ARG;
  VASMG_API_BEGIN
  Ctx& c = h->c;
  const double t0 = now_ms();
  join_user(c);
  int rc = solve_dev(c, F, U, tol, st);
  if (st) {
    st->solve_ms = now_ms() - t0;
    st->setup_ms = c.setup_ms;
    double nb0 = (double)c.C[0].nnzb, tot = 0;
    for (auto& l : c.C) tot += (double)l.nnzb;
    st->op_complexity = tot / nb0;
  }
  return rc;
  VASMG_API_END
}

int vasmg_solve_multi(vasmg_handle h, int32_t k, const double* const* F, double* const* U, double tol,
                      vasmg_stats* st) {
  if (!h || k < 0 || !(tol > 0.0) || (k > 0 && (!F || !U))) return VASMG_ERR_INVALID_ARG;
  for (int32_t i = 0; i < k; ++i)
    if (!F[i] || !U[i]) return VASMG_ERR_INVALID_ARG;
  if (k == 0) return VASMG_OK;
  VASMG_API_BEGIN
  Ctx& c = h->c;
  const double t0 = now_ms();
  join_user(c);
  const int rc = solve_multi_dev(c, k, F, U, tol, st);
  if (st) {
    const double ms = now_ms() - t0;
    double nb0 = (double)c.C[0].nnzb, tot = 0;
    for (auto& l : c.C) tot += (double)l.nnzb;
    for (int32_t i = 0; i < k; ++i) {
      st[i].solve_ms = ms;
      st[i].setup_ms = c.setup_ms;
      st[i].op_complexity = tot / nb0;
    }
  }
  return rc;
  VASMG_API_END
}

int vasmg_solve_batch(int32_t k, const vasmg_handle* h, const double* const* F, double* const* U, double tol,
                      vasmg_stats* st) {
  if (k < 0 || (k > 0 && (!h || !F || !U)) || !(tol > 0.0)) return VASMG_ERR_INVALID_ARG;
  for (int32_t i = 0; i < k; ++i)
    if (!h[i] || !F[i] || !U[i]) return VASMG_ERR_INVALID_ARG;
  // handles that can share launches: one launch per level and phase for all
  {
    int rc = -1000;
    const double t0 = now_ms();
    try {
      std::vector<Ctx*> cs;
      for (int32_t i = 0; i < k; ++i) cs.push_back(&h[i]->c);
      rc = solve_batch_dev(cs, F, U, tol, st, nullptr);
    } catch (const std::bad_alloc& e) {
      g_last_error = e.what();
      return VASMG_ERR_OOM;
    } catch (const std::exception& e) {
      return fail(e);
    }
    if (rc != -1000) {
      if (st) {
        const double ms = now_ms() - t0;
        for (int32_t i = 0; i < k; ++i) {
          const Ctx& c = h[i]->c;
          double nb0 = (double)c.C[0].nnzb, tot = 0;
          for (auto& l : c.C) tot += (double)l.nnzb;
          st[i].solve_ms = ms;
          st[i].setup_ms = c.setup_ms;
          st[i].op_complexity = tot / nb0;
        }
      }
      return rc;
    }
  }
  // groups of handles whose sweep grids are resident together
  int cap = 0;
  for (int32_t i = 0; i < k; ++i) {
    const int ci = h[i]->c.cta_capacity;
    if (ci > 0) cap = cap ? std::min(cap, ci) : ci;
  }
  std::vector<std::vector<int32_t>> groups;
  std::vector<int> load;
  for (int32_t i = 0; i < k; ++i) {
    const int need = std::max(1, h[i]->c.ctas_used);
    bool placed = false;
    if (!groups.empty()) {
      auto& g = groups.back();
      bool repeat = false;
      for (int32_t j : g) repeat = repeat || h[j] == h[i];
      if (!repeat && load.back() + need <= cap) {
        g.push_back(i);
        load.back() += need;
        placed = true;
      }
    }
    if (!placed) {
      groups.push_back({i});
      load.push_back(need);
    }
  }
  std::vector<int> rc(k, VASMG_OK);
  // each solve's error detail, taken in the thread that ran it (the detail
  // string is per thread) and handed to the caller's thread below
  std::vector<std::string> detail(k);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VASMG_ERR_CUDA;
  for (const auto& g : groups) {
    if (g.size() == 1) {
      const int32_t i = g[0];
      rc[i] = vasmg_solve(h[i], F[i], U[i], tol, st ? &st[i] : nullptr);
      if (rc[i] < 0) detail[i] = g_last_error;
      continue;
    }
    std::vector<std::thread> th;
    for (int32_t i : g)
      th.emplace_back([&, i]() {
        cudaSetDevice(dev);
        rc[i] = vasmg_solve(h[i], F[i], U[i], tol, st ? &st[i] : nullptr);
        if (rc[i] < 0) detail[i] = g_last_error;
      });
    for (auto& t : th) t.join();
  }
  int worst = VASMG_OK;
  for (int32_t i = 0; i < k; ++i) {
    if (rc[i] < 0) {
      g_last_error = "solve " + std::to_string(i) + " of the batch: " + detail[i];
      return rc[i];
    }
    worst = std::max(worst, rc[i]);
  }
  return worst;
}

int vasmg_num_levels(vasmg_handle h) {
  if (!h) return VASMG_ERR_INVALID_ARG;
  return (int)h->c.C.size();
}

int vasmg_level_info(vasmg_handle h, int32_t level, int64_t* n_vertices, int64_t* nnzb, int32_t* n_colours) {
  if (!h || level < 0 || level >= (int32_t)h->c.C.size()) return VASMG_ERR_INVALID_ARG;
  const CanonLevel& l = h->c.C[level];
  if (n_vertices) *n_vertices = l.nv;
  if (nnzb) *nnzb = l.nnzb;
  if (n_colours) *n_colours = l.ncol;
  return VASMG_OK;
}

int vasmg_export(vasmg_handle h, int32_t what, int32_t level, void* buf, int64_t* bytes) {
  if (!h || !bytes) return VASMG_ERR_INVALID_ARG;
  VASMG_API_BEGIN
  Ctx& c = h->c;
  const int d = c.dim;
  std::vector<char> out;
  auto put = [&](const void* p, size_t nbytes) {
    out.resize(nbytes);
    if (nbytes) std::memcpy(out.data(), p, nbytes);
  };
  auto dev = [&](const void* p, size_t nbytes) {
    out.resize(nbytes);
    if (nbytes) {
      VASMG_CUDA(cudaMemcpyAsync(out.data(), p, nbytes, cudaMemcpyDeviceToHost, c.stream));
      VASMG_CUDA(cudaStreamSynchronize(c.stream));
    }
  };
  auto widen = [&](const DevBuf<int32_t>& b) {
    std::vector<int32_t> v = b.download();
    std::vector<int64_t> w(v.begin(), v.end());
    put(w.data(), w.size() * 8);
  };
  const bool lvl_ok = level >= 0 && level < (int32_t)c.C.size();
  switch (what) {
    case VASMG_EXPORT_MORTON: dev(c.mkey.get(), (size_t)c.nv * 8); break;
    case VASMG_EXPORT_LEAF: {
      std::vector<u64> st = c.leaf_start.download();
      std::vector<uint8_t> dp = c.leaf_depth.download();
      std::vector<int64_t> w(2 * (size_t)c.nv);
      for (int64_t v = 0; v < c.nv; ++v) {
        w[2 * v] = dp[v];
        w[2 * v + 1] = (int64_t)(st[v] >> (d * (c.K - dp[v])));
      }
      put(w.data(), w.size() * 8);
      break;
    }
    case VASMG_EXPORT_BOX: {
      double b[2] = {c.box_m, c.box_M};
      put(b, 16);
      break;
    }
    case VASMG_EXPORT_LIFT: dev(c.lift.get(), (size_t)c.n * 8); break;
    case VASMG_EXPORT_VOL: dev(c.vol.get(), (size_t)c.ne * 8); break;
    case VASMG_EXPORT_LANES: {
      std::vector<int32_t> g(c.C.size(), 0);
      lanes_info(c, g.data(), (int)g.size());
      put(g.data(), g.size() * sizeof(int32_t));
      break;
    }
    case VASMG_EXPORT_STAGED: {
      VASMG_CHECK(lvl_ok, VASMG_ERR_INVALID_ARG, "level out of range");
      int64_t v[5];
      staged_info(c, level, v);
      put(v, sizeof(v));
      break;
    }
    case VASMG_EXPORT_DENSE: {
      int kd = -1, dn = 0;
      dense_level_info(c, &kd, &dn);
      int64_t v[2] = {kd, dn};
      put(v, 16);
      break;
    }
    default: {
      VASMG_CHECK(lvl_ok, VASMG_ERR_INVALID_ARG, "level out of range");
      CanonLevel& L = c.C[level];
      switch (what) {
        case VASMG_EXPORT_CELLS: {
          VASMG_CHECK(level >= 1, VASMG_ERR_INVALID_ARG, "cells exist on levels >= 1");
          std::vector<u64> st = L.cell_start.download();
          std::vector<uint8_t> dp = L.cell_depth.download();
          std::vector<int64_t> w(2 * st.size());
          for (size_t i = 0; i < st.size(); ++i) {
            w[2 * i] = dp[i];
            w[2 * i + 1] = (int64_t)(st[i] >> (d * (c.K - dp[i])));
          }
          put(w.data(), w.size() * 8);
          break;
        }
        case VASMG_EXPORT_LATTICE: dev(L.lat.get(), (size_t)L.lat.n * 8); break;
        case VASMG_EXPORT_P_RP: widen(L.prp); break;
        case VASMG_EXPORT_P_CI: dev(L.pci.get(), (size_t)L.pci.n * 4); break;
        case VASMG_EXPORT_P_W: dev(L.pw.get(), (size_t)L.pw.n * 8); break;
        case VASMG_EXPORT_A_RP: widen(L.rp); break;
        case VASMG_EXPORT_A_CI: dev(L.ci.get(), (size_t)L.ci.n * 4); break;
        case VASMG_EXPORT_A_V: dev(L.v.get(), (size_t)L.v.n * 8); break;
        case VASMG_EXPORT_DEAD: dev(L.dead.get(), (size_t)L.dead.n); break;
        case VASMG_EXPORT_COLOUR: dev(L.colour.get(), (size_t)L.colour.n * 4); break;
        case VASMG_EXPORT_DINV: dev(L.dinv.get(), (size_t)L.dinv.n * 8); break;
        default: throw Error(VASMG_ERR_INVALID_ARG, "unknown export selector");
      }
    }
  }
  *bytes = (int64_t)out.size();
  if (buf && !out.empty()) std::memcpy(buf, out.data(), out.size());
  return VASMG_OK;
  VASMG_API_END
}

int vasmg_apply(vasmg_handle h, int32_t op, int32_t level, const double* x, double* y) {
  if (!h || !x || !y) return VASMG_ERR_INVALID_ARG;
  VASMG_API_BEGIN
  Ctx& c = h->c;
  VASMG_CHECK(level >= 0 && level < (int32_t)c.C.size(), VASMG_ERR_INVALID_ARG, "level out of range");
  join_user(c);
  const int d = c.dim;
  const int L = (int)c.C.size();
  i64 nx = c.C[level].nv * d, ny = nx;
  if (op == VASMG_OP_RESTRICT) {
    VASMG_CHECK(level + 1 < L, VASMG_ERR_INVALID_ARG, "no coarser level");
    ny = c.C[level + 1].nv * d;
  }
  if (op == VASMG_OP_PROLONG) {
    VASMG_CHECK(level + 1 < L, VASMG_ERR_INVALID_ARG, "no coarser level");
    nx = c.C[level + 1].nv * d;
  }
  if (op == VASMG_OP_COARSE) nx = ny = c.C[L - 1].nv * d;
  DevBuf<double> dx, dy;
  dx.alloc(nx, c.stream);
  dy.alloc(ny, c.stream);
  VASMG_CUDA(cudaMemcpyAsync(dx.get(), x, sizeof(double) * nx, cudaMemcpyDefault, c.stream));
  VASMG_CUDA(cudaMemcpyAsync(dy.get(), y, sizeof(double) * ny, cudaMemcpyDefault, c.stream));
  apply_op(c, op, level, dx.get(), dy.get());
  VASMG_CUDA(cudaMemcpyAsync(y, dy.get(), sizeof(double) * ny, cudaMemcpyDefault, c.stream));
  VASMG_CUDA(cudaStreamSynchronize(c.stream));
  return VASMG_OK;
  VASMG_API_END
}

int vasmg_time_kernel(vasmg_handle h, int32_t which, int32_t level, int32_t reps, double* ms, double* bytes) {
  if (!h || !ms || !bytes || reps <= 0) return VASMG_ERR_INVALID_ARG;
  if (level < 0 || level >= (int32_t)h->c.C.size()) return VASMG_ERR_INVALID_ARG;
  VASMG_API_BEGIN
  join_user(h->c);
  *ms = time_kernel(h->c, which, level, reps, bytes);
  return VASMG_OK;
  VASMG_API_END
}

int vasmg_time_kernel_multi(vasmg_handle h, int32_t which, int32_t level, int32_t k, int32_t reps, double* ms,
                            double* bytes) {
  if (!h || !ms || !bytes || reps <= 0 || (k != 2 && k != 4 && k != 8)) return VASMG_ERR_INVALID_ARG;
  if (level < 0 || level >= (int32_t)h->c.C.size()) return VASMG_ERR_INVALID_ARG;
  VASMG_API_BEGIN
  join_user(h->c);
  *ms = time_kernel_multi(h->c, which, level, k, reps, bytes);
  return VASMG_OK;
  VASMG_API_END
}

int vasmg_coarse_solve_noalloc(vasmg_handle h, const double* b, double* x, void* stream) {
  if (!h || !b || !x) return VASMG_ERR_INVALID_ARG;
  const Ctx& c = h->c;
  const i64 n = c.nc;
  if (n <= 0 || n > VASMG_NOALLOC_MAX_DOFS) return VASMG_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VASMG_ERR_CUDA;
  // the factor lives on the handle's device: the kernel must run there
  if (dev != c.device) return VASMG_ERR_INVALID_ARG;
  if (!on_device(b, dev) || !on_device(x, dev)) return VASMG_ERR_INVALID_ARG;
  double* scratch = nullptr;
  {
    const unsigned long long ctx = current_ctx_id();
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocSlot& slot = g_noalloc_slot[dev];
    if (!slot.ptr || slot.ctx_id != ctx || ctx == 0) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return VASMG_ERR_CUDA;
      }
      slot.ptr = (double*)p;
      slot.ctx_id = ctx;
    }
    scratch = slot.ptr;
  }
  cudaStream_t s = (cudaStream_t)stream;
  coarse_noalloc_kernel<<<1, 32, 0, s>>>(c.chol.get(), c.chol_drop.get(), (int)n, b, x, scratch);
  if (cudaGetLastError() != cudaSuccess) return VASMG_ERR_CUDA;
  // vasmg_update_data waits for this before it refills the factor
  if (cudaEventRecord(c.noalloc_ev, s) != cudaSuccess) {
    cudaGetLastError();
    return VASMG_ERR_CUDA;
  }
  return VASMG_OK;
}

int64_t vasmg_last_launch_count(vasmg_handle h) { return h ? h->c.last_launches : -1; }

int vasmg_destroy(vasmg_handle h) {
  if (!h) return VASMG_ERR_INVALID_ARG;
  VASMG_API_BEGIN
  destroy_ctx(h);
  return VASMG_OK;
  VASMG_API_END
}

const char* vasmg_error_string(int code) {
  switch (code) {
    case VASMG_OK: return "ok";
    case VASMG_NOT_CONVERGED: return "not converged within max_iters";
    case VASMG_ERR_INVALID_ARG: return "invalid argument";
    case VASMG_ERR_DEGENERATE_ELEMENT: return "degenerate element (zero or non-finite measure)";
    case VASMG_ERR_OOM: return "out of device memory";
    case VASMG_ERR_CUDA: return "CUDA error";
    case VASMG_ERR_BREAKDOWN: return "PCG breakdown (p^T q <= 0 or NaN)";
    case VASMG_ERR_TIMEOUT: return "a bounded device wait gave up";
    case VASMG_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
  }
}

// Detail of the last error on this thread (not part of the stable ABI).
const char* vasmg_last_error_detail(void) { return g_last_error.c_str(); }

int vasmg_probe_fp64_rate(double* tflops, double* ms) {
  if (!tflops) return VASMG_ERR_INVALID_ARG;
  VASMG_API_BEGIN
  return probe_fp64_rate(tflops, ms);
  VASMG_API_END
}

int vasmg_probe_wait_timeout(double* elapsed_ms) {
  VASMG_API_BEGIN
  return probe_wait_timeout(elapsed_ms);
  VASMG_API_END
}

}  // extern "C"
