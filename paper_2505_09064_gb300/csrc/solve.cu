// The hot path: one PCG iteration (Alg. 2) preconditioned by one V-cycle
// (Alg. 3, recursive) of V-ASMG.
//
// Outer CG, FP64, level-0 solve order:
//   spmv_sell    q = A p with A in SELL-32 (slices of 32 rows, one thread per
//                row, diagonal block included), p.q, alpha = rho / p.q.  GB300
//                runs FP64 at a small fraction of its FP32 rate, so the layout
//                keeps every lane's DFMA useful;
//   cg_update    U += alpha p, r -= alpha q, ||r||, stop test ||r||/||F|| < tol
//                (Sec. 5 item (3)), b_0 = r cast to the V-cycle precision;
//   rz           rho_new = r.z, beta = rho_new / rho;   p_update  p = z + beta p.
// Reductions are deterministic: every block writes one partial and the last
// block to finish sums the partials in index order.
//
// V-cycle (precision V, operator values stored as S).  For each level with
// more than TAIL_NV vertices, five launches:
//   vdown     forward multicolour block Gauss-Seidel sweep from a zero initial
//             guess, x_i = D_ii^{-1}(b_i - sum_{j of an earlier colour} A_ij x_j)
//             (with a zero start the later colours contribute nothing, so only
//             the "lower" part of each row is read, from its own arrays);
//   residual  r_i = - sum_{j of a later colour} A_ij x_j (b_i - A_ii x_i - lower
//             is exactly zero after the sweep), the "upper" part only;
//   restrict  b_{l+1} = P^T r (eq. (R));
//   prolong   x_l += P x_{l+1} (masked at dead dofs);
//   vup       backward sweep (colours in reverse order) with full rows.
// The two sweeps are cooperative launches with one CTA per region (a range of
// spatial keys, one contiguous row range per colour).  A region runs its
// colours in order; before a colour it waits until every neighbouring region
// has published the stage it reads (64-bit epoch/stage words, release /
// acquire at GPU scope).  Every wait is bounded; a wait that gives up raises a
// global abort flag and the solve returns VASMG_ERR_TIMEOUT.  The last CTA to
// leave a launch advances its epoch.  Residual, restriction and prolongation
// have no dependencies within themselves and run as plain kernels.  The
// lanes per row G of each such level are timed at setup (autotune) or set by
// rule from the mean row length.
//
// Levels with at most TAIL_NV vertices and the coarsest Cholesky solve run in
// one thread-block-cluster kernel (hardware cluster barriers between phases;
// the smallest levels on CTA 0 alone with their vectors in shared memory).
// With FP32 vectors, the V-cycle from a small level k down is a fixed linear
// map that setup precomputes as a dense matrix (the cycle applied to the unit
// vectors); the tail then applies it as x_k = M b_k on the whole cluster
// instead of recursing below k.
//
// The whole solve is one CUDA graph with a conditional WHILE node (no host
// round trip per iteration).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "solve_dev.cuh"

namespace vasmg {

// ------------------------------------------------------------------ setup kernels for the engine

// Copy each row's lower (earlier-colour) and upper (later-colour) blocks into
// separate contiguous arrays: row i's lower entries start at rpl[i], its upper
// entries at rph[i].
template <typename S>
__global__ void split_parts_kernel(const int* __restrict__ rp, const int* __restrict__ sp,
                                   const int* __restrict__ ci, const S* __restrict__ off, long long nnz, int dd,
                                   int nv, const int* __restrict__ rpl, const int* __restrict__ rph,
                                   int* __restrict__ cil, S* __restrict__ offl, long long nlo,
                                   int* __restrict__ cih, S* __restrict__ offh, long long nhi) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    const int k0 = rp[i], ks = sp[i], k1 = rp[i + 1];
    for (int k = k0; k < ks; ++k) {
      const long long d = rpl[i] + (k - k0);
      cil[d] = ci[k];
      for (int q = 0; q < dd; ++q) offl[block_index(q, d, nlo, dd)] = off[block_index(q, k, nnz, dd)];
    }
    for (int k = ks; k < k1; ++k) {
      const long long d = rph[i] + (k - ks);
      cih[d] = ci[k];
      for (int q = 0; q < dd; ++q) offh[block_index(q, d, nhi, dd)] = off[block_index(q, k, nnz, dd)];
    }
  }
}

// SELL-32: rows sorted by length (longest first) inside windows of 1024 rows
__global__ void sell_keys_kernel(const int* __restrict__ rp, int nv, u64* __restrict__ keys, int* __restrict__ vals) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nv; r += gridDim.x * blockDim.x) {
    const u64 len = (u64)(rp[r + 1] - rp[r] + 1);  // + diagonal
    keys[r] = ((u64)(r >> 10) << 40) | ((1023ull - len) << 30) | (u64)(r & 1023);
    vals[r] = r;
  }
}

__global__ void sell_width_kernel(const int* __restrict__ rows, const int* __restrict__ rp, long long nslices,
                                  int nv, int* __restrict__ w, long long* __restrict__ wbytes) {
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < nslices;
       s += (long long)gridDim.x * blockDim.x) {
    int m = 0;
    for (int l = 0; l < 32; ++l) {
      const long long i = s * 32 + l;
      if (i < nv) {
        const int r = rows[i];
        m = max(m, rp[r + 1] - rp[r] + 1);
      }
    }
    w[s] = m;
    wbytes[s] = (long long)m * 32;
  }
}

template <int D>
__global__ void sell_fill_kernel(const int* __restrict__ rows, const int* __restrict__ rp, const int* __restrict__ ci,
                                 const double* __restrict__ off, long long nnz, const double* __restrict__ diag, int nv,
                                 long long nslices, const long long* __restrict__ ptr, const int* __restrict__ w,
                                 long long tot, int* __restrict__ sci, double* __restrict__ sv,
                                 int* __restrict__ srow) {
  constexpr int DD = D * D;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nslices * 32;
       i += (long long)gridDim.x * blockDim.x) {
    const long long s = i >> 5;
    const int lane = (int)(i & 31);
    const int r = i < nv ? rows[i] : -1;
    srow[i] = r;
    const int width = w[s];
    for (int k = 0; k < width; ++k) {
      const long long idx = ptr[s] + (long long)k * 32 + lane;
      int col;
      double blk[DD];
      if (r < 0) {
        col = 0;
        for (int q = 0; q < DD; ++q) blk[q] = 0.0;
      } else if (k == 0) {
        col = r;
        for (int q = 0; q < DD; ++q) blk[q] = diag[(long long)q * nv + r];
      } else if (rp[r] + k - 1 < rp[r + 1]) {
        const long long e = rp[r] + k - 1;
        col = ci[e];
        for (int q = 0; q < DD; ++q) blk[q] = off[block_index(q, e, nnz, DD)];
      } else {
        col = r;
        for (int q = 0; q < DD; ++q) blk[q] = 0.0;
      }
      sci[idx] = col;
      for (int q = 0; q < DD; ++q) sv[(long long)q * tot + idx] = blk[q];
    }
  }
}

// ------------------------------------------------------------------ cycle variants (W-cycle, additive form)

// out = bs - A x on one level, every block of each row (the diagonal one from
// the FP64 diagonal planes): the coarse residual on which the W-cycle's
// second coarse cycle runs.  G lanes per row as in the residual kernel.
template <int D, int G, typename V, typename S>
__global__ void __launch_bounds__(256) full_residual_kernel(const __grid_constant__ LV<V> L,
                                                            const double* __restrict__ diag,
                                                            const V* __restrict__ bs, V* __restrict__ out) {
  constexpr int NG = 256 / G;
  const int g = threadIdx.x / G, lane = threadIdx.x & (G - 1);
  for (int base = blockIdx.x * NG; base < L.nv; base += gridDim.x * NG) {
    const int row = base + g;
    const bool valid = row < L.nv;
    RowSeg sg{0, 0, 0, 0};
    if (valid) sg = seg_range<1>(L, row);
    V acc[D];
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] = V(0);
    row_entries<D, G, V, S, 1, false, true>(L, sg, lane, acc);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o, G);
    if (valid && lane < D) {
      V dx = V(0);
#pragma unroll
      for (int bb = 0; bb < D; ++bb)
        dx += (V)__ldg(diag + (long long)(lane * D + bb) * L.nv + row) * __ldcg((const V*)L.x + (long long)row * D + bb);
      out[(long long)row * D + lane] = bs[(long long)row * D + lane] - (pick<D>(acc, lane) + dx);
    }
  }
}

template <typename V>
__global__ void vcopy_kernel(V* __restrict__ dst, const V* __restrict__ src, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    dst[t] = src[t];
}

template <typename V>
__global__ void vadd_kernel(V* __restrict__ dst, const V* __restrict__ src, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    dst[t] += src[t];
}

// ------------------------------------------------------------------ conversions for vasmg_apply

template <typename V>
__global__ void to_solve_kernel(const double* __restrict__ in, V* __restrict__ out, const int* __restrict__ perm,
                                long long nv, int d) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nv * d;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / d;
    out[t] = (V)in[(long long)perm[r] * d + (t - r * d)];
  }
}
template <typename V>
__global__ void from_solve_kernel(const V* __restrict__ in, double* __restrict__ out, const int* __restrict__ perm,
                                  long long nv, int d) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nv * d;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / d;
    out[(long long)perm[r] * d + (t - r * d)] = (double)in[t];
  }
}

// ------------------------------------------------------------------ engine

// Lengths of each row's lower (earlier-colour) and upper parts; entry nv is
// 0 so that exclusive scans of the n + 1 entries end with the totals.
__global__ void part_lengths_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ sp, int nv,
                                    int32_t* __restrict__ nlo, int32_t* __restrict__ nhi) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nv; i += gridDim.x * blockDim.x) {
    nlo[i] = i < nv ? sp[i] - rp[i] : 0;
    nhi[i] = i < nv ? rp[i + 1] - sp[i] : 0;
  }
}

// Region adjacency bits: for every block (i, j) of a row i in region k whose
// column j lies in region k2 != k, bit k2 of region k's W words.  A word
// already holding the bit is not written again.
__global__ void region_bits_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int nv,
                                   const int32_t* __restrict__ reg, int W, unsigned long long* bits) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    const int k = reg[i];
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int k2 = reg[ci[e]];
      if (k2 == k) continue;
      unsigned long long* w = bits + (long long)k * W + (k2 >> 6);
      const unsigned long long m = 1ull << (k2 & 63);
      if (!(*(volatile unsigned long long*)w & m)) atomicOr(w, m);
    }
  }
}

struct EngineBase {
  virtual ~EngineBase() {}
  virtual int solve(Ctx& c, const double* F, double* U, double tol, vasmg_stats* st) = 0;
  virtual void apply(Ctx& c, int op, int level, const double* x, double* y) = 0;
  virtual double time(Ctx& c, int which, int level, int reps, double* bytes) = 0;
  // refill the engine's own copies of operator values (same structure)
  virtual void refresh_values() = 0;
  // the dense level and the order of its matrix, (-1, 0) if none
  virtual void dense_level(int* k, int* n) const = 0;
  // lanes per row of the region levels (levels below the tail), 0 elsewhere
  virtual void lanes(int32_t* g, int n) const = 0;
  // level l's staged sweep copies: (forward slots, lower-part blocks,
  // backward slots, whole-row blocks, bytes per slot); zeros if unstaged
  virtual void staged(int l, int64_t* v) const = 0;
  // k right-hand sides on this hierarchy (solve_multi.cu for the FP32-vector modes)
  virtual int solve_multi(Ctx& c, int k, const double* const* F, double* const* U, double tol, vasmg_stats* st) = 0;
  virtual double time_multi(Ctx& c, int which, int level, int k, int reps, double* bytes) = 0;
  // the engine's view for a batched launch; false unless the V-cycle has FP32
  // vectors and is the plain V-cycle
  virtual bool batch_view(EngineView<float>* v) = 0;
  virtual int storage() const = 0;  // 0 FP64, 1 FP32, 2 BF16 operator values
};

// Lanes per row measured rather than picked by rule (vasmg_options.autotune):
// G changes the order of additions within a row, so a level's choice is kept
// per level signature for the whole process, and every handle of the same
// problem sweeps with the same G and gives the same bits.
struct LaneKey {
  int d, precision;
  long long nv, nnz;
  bool operator<(const LaneKey& o) const {
    return std::tie(d, precision, nv, nnz) < std::tie(o.d, o.precision, o.nv, o.nnz);
  }
};
static std::mutex& lane_cache_mutex() {
  static std::mutex m;
  return m;
}
static std::map<LaneKey, int>& lane_cache() {
  static std::map<LaneKey, int> m;
  return m;
}

// Lanes per row: few enough that a CTA pass covers many rows (the sweeps are
// bound by the latency of their dependent loads, not by lane utilisation).
static int pick_G(double avg) {
  if (avg <= 6.0) return 4;
  if (avg <= 48.0) return 8;
  if (avg <= 64.0) return 16;
  return 32;
}

template <int D, typename V, typename S>
struct Engine : EngineBase {
  Ctx* c = nullptr;
  int L = 0;       // number of levels
  int lt = 0;      // first tail level
  int nct = 1;     // CTAs in the tail cluster
  int kd = -1;     // dense level (FP32 vectors): x_kd = M b_kd replaces the cycle below it
  int dn = 0;      // order of M
  int dld = 0;     // row stride of M (dn rounded up to a multiple of 4)
  DevBuf<V> dm;    // M, row-major, zero-padded columns
  int sms_ = 1;    // SMs of the device
  std::vector<LV<V>> lv;
  std::vector<int> G;
  std::vector<DevBuf<int32_t>> cs_dev, rs_dev, nb_rp, nb;
  std::vector<DevBuf<unsigned long long>> pg_d, pg_u;
  std::vector<i64> nnz_lo;        // lower-part (earlier colour) blocks per level
  std::vector<DevBuf<int32_t>> rpl_dev, rph_dev, cil_dev, cih_dev;
  std::vector<DevBuf<S>> offl_dev, offh_dev;
  DevBuf<int> ctrs;
  DevBuf<double> coarse_y;
  // CG
  DevBuf<double> U, r, p, q, part, hist, Fbuf, Ubuf;
  DevBuf<Scalars> sc;
  DevBuf<int32_t> sell_rows, sell_w, sell_ci;
  DevBuf<int32_t> sell_order;     // level-0 rows sorted by length (SELL fill order)
  DevBuf<long long> sell_ptr;
  DevBuf<double> sell_v;
  i64 sell_real_entries = 0;
  Scalars* host_sc = nullptr;
  CGArgs cga{};
  int cg_blocks = 0, spmv_blocks = 0;
  CoarseArgs co{};
  // graphs
  cudaGraphExec_t exec_while = nullptr;
  cudaGraphExec_t exec_body = nullptr;
  i64 launches_body = 0;
  i64 launch_counter = 0;
  MultiBase* multi = nullptr;  // several right-hand sides (FP32-vector modes), made on first use
  // gamma-cycle (gamma >= 2): each level's coarse right-hand side and first
  // coarse correction, kept while the next coarse cycle runs
  std::vector<DevBuf<V>> wb, we;
  // 3D region levels: the sweeps' operator parts in the staged order
  // (vstaged_kernel), [0] the forward sweep's lower part, [1] the backward
  // sweep's whole rows, each built for the level's lanes per row G
  struct Staged {
    int G = 0;                  // 0: not built
    long long nslots = 0;
    DevBuf<int32_t> ci, goff, srow, step_nact;
    DevBuf<long long> step_off;
    DevBuf<S> v8, v9;
    StagedOp<S> op{};
  };
  std::vector<Staged> stg[2];

  explicit Engine(Ctx& ctx) : c(&ctx) { build(); }
  ~Engine() override {
    delete multi;
    if (exec_while) cudaGraphExecDestroy(exec_while);
    if (exec_body) cudaGraphExecDestroy(exec_body);
    if (host_sc) cudaFreeHost(host_sc);
  }

  const void* off_ptr(SolveLevel& s) {
    if (std::is_same<S, double>::value) return s.off64.get();
    if (std::is_same<S, float>::value) return s.off32.get();
    return s.off16.get();
  }
  const V* dinv_ptr(SolveLevel& s) {
    if (std::is_same<V, double>::value) return (const V*)s.dinv64.get();
    return (const V*)s.dinv32.get();
  }
  const V* pw_ptr(SolveLevel& s) {
    if (std::is_same<V, double>::value) return (const V*)s.pw64.get();
    return (const V*)s.pw32.get();
  }
  const V* rw_ptr(SolveLevel& s) {
    if (std::is_same<V, double>::value) return (const V*)s.rw64.get();
    return (const V*)s.rw32.get();
  }

  // Regions of one level.  The spatial keys (Morton rank of a fine vertex,
  // lattice Morton order of a coarse one) are a permutation of 0..nv-1 and
  // ascend within each colour, so region k (keys [k nv/R, (k+1) nv/R)) owns
  // one contiguous row range per colour.
  void build_regions(int l, int R) {
    cudaStream_t s = c->stream;
    SolveLevel& sl = c->S[l];
    const int nv = (int)sl.nv, C = sl.ncol;
    VASMG_CHECK((int)sl.sec.size() == nv, VASMG_ERR_UNSUPPORTED, "missing spatial keys");
    std::vector<int> RS((size_t)C * (R + 1));
    std::vector<int> reg(nv);
    for (int col = 0; col < C; ++col) {
      const auto b0 = sl.sec.begin() + sl.cs[col], b1 = sl.sec.begin() + sl.cs[col + 1];
      for (int k = 0; k <= R; ++k) {
        const uint32_t key = (uint32_t)((i64)k * nv / R);
        RS[(size_t)col * (R + 1) + k] = (int)(std::lower_bound(b0, b1, key) - sl.sec.begin());
      }
      for (int k = 0; k < R; ++k)
        for (int i = RS[(size_t)col * (R + 1) + k]; i < RS[(size_t)col * (R + 1) + k + 1]; ++i) reg[i] = k;
    }
    const int W = (R + 63) / 64;
    auto to_csr = [&](const std::vector<u64>& bits, DevBuf<int32_t>& rp_d, DevBuf<int32_t>& list_d) {
      std::vector<int> rp(R + 1, 0), list;
      for (int k = 0; k < R; ++k) {
        for (int w = 0; w < W; ++w)
          for (u64 m = bits[(size_t)k * W + w]; m; m &= m - 1) list.push_back(w * 64 + __builtin_ctzll(m));
        rp[k + 1] = (int)list.size();
      }
      if (list.empty()) list.push_back(0);
      rp_d.alloc(R + 1, s);
      rp_d.upload(rp.data(), R + 1);
      list_d.alloc((i64)list.size(), s);
      list_d.upload(list.data(), (i64)list.size());
    };
    {
      // the blocks split by part (lower / upper), each part contiguous: row
      // pointers by exclusive scans of the part lengths, on the device
      rpl_dev[l].alloc(nv + 1, s);
      rph_dev[l].alloc(nv + 1, s);
      part_lengths_kernel<<<grid_for(nv + 1, 256), 256, 0, s>>>(sl.rp.get(), sl.sp.get(), nv, rpl_dev[l].get(),
                                                                 rph_dev[l].get());
      check_launch("part_lengths");
      scan_exclusive_i32(rpl_dev[l].get(), rpl_dev[l].get(), nv + 1, s);
      scan_exclusive_i32(rph_dev[l].get(), rph_dev[l].get(), nv + 1, s);
      const i64 lo = fetch(rpl_dev[l].get() + nv, s);
      nnz_lo[l] = lo;
      {
        const i64 hi = sl.nnz - lo;
        cil_dev[l].alloc(std::max<i64>(lo, 1), s);
        cih_dev[l].alloc(std::max<i64>(hi, 1), s);
        offl_dev[l].alloc(std::max<i64>((i64)D * D * lo, 1), s);
        offh_dev[l].alloc(std::max<i64>((i64)D * D * hi, 1), s);
        if (nv > 0) {
          split_parts_kernel<S><<<grid_for(nv, 256), 256, 0, s>>>(
              sl.rp.get(), sl.sp.get(), sl.ci.get(), (const S*)off_ptr(sl), sl.nnz, D * D, nv, rpl_dev[l].get(),
              rph_dev[l].get(), cil_dev[l].get(), offl_dev[l].get(), lo, cih_dev[l].get(), offh_dev[l].get(), hi);
          check_launch("split_parts");
        }
        LV<V>& v = lv[l];
        v.rpl = rpl_dev[l].get();
        v.cil = cil_dev[l].get();
        v.offl = offl_dev[l].get();
        v.nlo = lo;
        v.rph = rph_dev[l].get();
        v.cih = cih_dev[l].get();
        v.offh = offh_dev[l].get();
        v.nhi = hi;
      }
      // region adjacency: bit k2 of region k's words for every block (i, j)
      // with i in region k and j in region k2 != k, set on the device
      DevBuf<int32_t> reg_d;
      reg_d.alloc(std::max(nv, 1), s);
      reg_d.upload(reg.data(), nv);
      DevBuf<u64> bits_d;
      bits_d.alloc((i64)R * W, s);
      bits_d.zero();
      if (nv > 0) {
        region_bits_kernel<<<grid_for(nv, 256), 256, 0, s>>>(sl.rp.get(), sl.ci.get(), nv, reg_d.get(), W,
                                                             (unsigned long long*)bits_d.get());
        check_launch("region_bits");
      }
      to_csr(bits_d.download(), nb_rp[l], nb[l]);
    }
    rs_dev[l].alloc((i64)RS.size(), s);
    rs_dev[l].upload(RS.data(), (i64)RS.size());
    pg_d[l].alloc(R, s);
    pg_u[l].alloc(R, s);
    pg_d[l].zero();
    pg_u[l].zero();
    LV<V>& v = lv[l];
    v.R = R;
    v.RS = rs_dev[l].get();
    v.nb_rp = nb_rp[l].get();
    v.nb = nb[l].get();
    v.pg_d = pg_d[l].get();
    v.pg_u = pg_u[l].get();
  }

  // New operator values on the same structure: the level-0 FP64 SELL copy
  // and the split lower / upper parts of every level are refilled in place.
  void refresh_values() override {
    cudaStream_t s = c->stream;
    SolveLevel& s0 = c->S[0];
    const int nv = (int)s0.nv;
    const long long nslices = ceil_div(nv, 32);
    sell_fill_kernel<D><<<grid_for(nslices * 32, 256), 256, 0, s>>>(
        sell_order.get(), s0.rp.get(), s0.ci.get(), s0.off64.get(), s0.nnz, s0.diag64.get(), nv, nslices,
        sell_ptr.get(), sell_w.get(), cga.sell_tot, sell_ci.get(), sell_v.get(), sell_rows.get());
    check_launch("sell_fill");
    for (int l = 0; l + 1 < L; ++l) {
      SolveLevel& sl = c->S[l];
      if (sl.nv == 0) continue;
      split_parts_kernel<S><<<grid_for(sl.nv, 256), 256, 0, s>>>(
          sl.rp.get(), sl.sp.get(), sl.ci.get(), (const S*)off_ptr(sl), sl.nnz, D * D, (int)sl.nv, rpl_dev[l].get(),
          rph_dev[l].get(), cil_dev[l].get(), offl_dev[l].get(), lv[l].nlo, cih_dev[l].get(), offh_dev[l].get(),
          lv[l].nhi);
      check_launch("split_parts");
      fill_staged(l, 0);
      fill_staged(l, 1);
    }
    build_dense_level();
    VASMG_CUDA(cudaStreamSynchronize(s));
  }

  void build_sell() {
    cudaStream_t s = c->stream;
    SolveLevel& s0 = c->S[0];
    const int nv = (int)s0.nv;
    DevBuf<u64> keys;
    keys.alloc(nv, s);
    DevBuf<int32_t>& rows = sell_order;
    rows.alloc(nv, s);
    sell_keys_kernel<<<grid_for(nv, 256), 256, 0, s>>>(s0.rp.get(), nv, keys.get(), rows.get());
    check_launch("sell_keys");
    radix_sort(keys.get(), rows.get(), nv, 64, s);
    const long long nslices = ceil_div(nv, 32);
    sell_w.alloc(nslices, s);
    DevBuf<long long> wb;
    wb.alloc(nslices + 1, s);
    wb.zero();
    sell_width_kernel<<<grid_for(nslices, 256), 256, 0, s>>>(rows.get(), s0.rp.get(), nslices, nv, sell_w.get(),
                                                             wb.get());
    check_launch("sell_width");
    scan_exclusive_i64((const i64*)wb.get(), (i64*)wb.get(), nslices + 1, s);
    const long long tot = fetch(wb.get() + nslices, s);
    sell_ptr = std::move(wb);
    sell_ci.alloc(tot, s);
    sell_v.alloc((i64)D * D * tot, s);
    sell_rows.alloc(nslices * 32, s);
    sell_fill_kernel<D><<<grid_for(nslices * 32, 256), 256, 0, s>>>(
        rows.get(), s0.rp.get(), s0.ci.get(), s0.off64.get(), s0.nnz, s0.diag64.get(), nv, nslices, sell_ptr.get(),
        sell_w.get(), tot, sell_ci.get(), sell_v.get(), sell_rows.get());
    check_launch("sell_fill");
    sell_real_entries = s0.nnz + s0.nv;
    cga.sell_n = nslices * 32;
    cga.sell_tot = tot;
    cga.sell_rows = sell_rows.get();
    cga.sell_ptr = sell_ptr.get();
    cga.sell_w = sell_w.get();
    cga.sell_ci = sell_ci.get();
    cga.sell_v = sell_v.get();
  }

  void build() {
    cudaStream_t s = c->stream;
    L = (int)c->S.size();
    VASMG_CHECK(L <= MAX_LEVELS, VASMG_ERR_UNSUPPORTED, "too many levels");
    lv.assign(L, LV<V>{});
    G.resize(L);
    cs_dev.resize(L);
    rs_dev.resize(L);
    nb_rp.resize(L);
    nb.resize(L);
    pg_d.resize(L);
    pg_u.resize(L);
    nnz_lo.assign(L, 0);
    rpl_dev.resize(L);
    rph_dev.resize(L);
    cil_dev.resize(L);
    cih_dev.resize(L);
    offl_dev.resize(L);
    offh_dev.resize(L);
    ctrs.alloc((i64)L * C_N, s);
    {
      std::vector<int> h((size_t)L * C_N, 0);
      for (int l = 0; l < L; ++l) {
        h[l * C_N + C_DEPOCH] = 1;
        h[l * C_N + C_UEPOCH] = 1;
      }
      ctrs.upload(h.data(), (i64)L * C_N);
    }
    for (int l = 0; l < L; ++l) {
      SolveLevel& sl = c->S[l];
      const i64 n = sl.nv * D;
      sl.x.alloc(n * sizeof(V), s);
      sl.b.alloc(n * sizeof(V), s);
      sl.r.alloc(n * sizeof(V), s);
      sl.x.zero();
      sl.b.zero();
      sl.r.zero();
      cs_dev[l].alloc(sl.ncol + 1, s);
      cs_dev[l].upload(sl.cs.data(), sl.ncol + 1);
      LV<V>& v = lv[l];
      v.nv = (int)sl.nv;
      v.ncol = sl.ncol;
      v.nnz = sl.nnz;
      v.rp = sl.rp.get();
      v.ci = sl.ci.get();
      v.sp = sl.sp.get();
      v.off = off_ptr(sl);
      v.dinv = dinv_ptr(sl);
      v.dead = sl.deadbits.get();
      v.x = (V*)sl.x.get();
      v.b = (V*)sl.b.get();
      v.r = (V*)sl.r.get();
      v.cs = cs_dev[l].get();
      v.ctr = ctrs.get() + (i64)l * C_N;
      G[l] = pick_G(sl.nv > 0 ? (double)sl.nnz / (double)sl.nv : 1.0);
    }
    for (int l = 0; l + 1 < L; ++l) {
      SolveLevel& sl = c->S[l];
      LV<V>& v = lv[l];
      v.nvc = (int)c->S[l + 1].nv;
      v.prp = sl.prp.get();
      v.pci = sl.pci.get();
      v.pw = pw_ptr(sl);
      v.rrp = sl.rrp.get();
      v.rci = sl.rci.get();
      v.rw = rw_ptr(sl);
      v.bc = lv[l + 1].b;
      v.xc = lv[l + 1].x;
    }
    lt = L - 1;
    while (lt > 0 && c->S[lt - 1].nv <= TAIL_NV) --lt;
    // one region per co-resident CTA (the launches are cooperative), at
    // least REGION_MIN_ROWS rows per region
    int dev = 0, sms = 0;
    VASMG_CUDA(cudaGetDevice(&dev));
    VASMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    sms_ = sms;
    for (int l = 0; l + 1 < L; ++l) {
      int bd = 1, bu = 1;
      switch (G[l]) {
        case 4: occ<4>(&bd, &bu); break;
        case 8: occ<8>(&bd, &bu); break;
        case 16: occ<16>(&bd, &bu); break;
        default: occ<32>(&bd, &bu); break;
      }
      const i64 cap = (i64)std::min(bd, bu) * sms;
      VASMG_CHECK(cap >= 1, VASMG_ERR_CUDA, "sweep kernel cannot be resident");
      i64 lim = cap;
      if (c->max_ctas > 0) lim = std::min<i64>(lim, c->max_ctas);
      const int R = (int)std::max<i64>(1, std::min<i64>(lim, ceil_div(c->S[l].nv, REGION_MIN_ROWS)));
      build_regions(l, R);
      c->ctas_used = std::max(c->ctas_used, R);
      c->cta_capacity = c->cta_capacity ? std::min<int>(c->cta_capacity, (int)cap) : (int)cap;
    }
    VASMG_CUDA(cudaFuncSetAttribute(tail_kernel<D, V, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, TAIL_SMEM_MAX));
    staged_attrs<4>();
    staged_attrs<8>();
    staged_attrs<16>();
    staged_attrs<32>();
    stg[0].resize(L);
    stg[1].resize(L);
    if constexpr (std::is_same<V, float>::value)
      VASMG_CUDA(cudaFuncSetAttribute(dense_level_kernel<D, V, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TAIL_SMEM_MAX));
    // tail cluster size: as many CTAs (<= 16) as the work of the tail levels warrants
    {
      i64 work = 0;
      for (int l = lt; l < L; ++l) work += c->S[l].nnz;
      nct = 1;
      while (nct < 16 && work > (i64)nct * 4 * TAIL_THREADS * 8) nct *= 2;
      if (nct > 8)
        if (cudaFuncSetAttribute(tail_kernel<D, V, S>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess)
          nct = 8;
      cudaGetLastError();
      while (nct > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nct);
        cfg.blockDim = dim3(TAIL_THREADS);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = nct;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, tail_kernel<D, V, S>, &cfg) == cudaSuccess && nclusters > 0)
          break;
        cudaGetLastError();
        nct /= 2;
      }
    }
    // coarsest
    coarse_y.alloc(c->nc, s);
    co.chol = c->chol.get();
    co.drop = c->chol_drop.get();
    co.perm = c->S[L - 1].perm.get();
    co.y = coarse_y.get();
    co.n = (int)c->nc;
    co.d = D;
    build_dense_level();
    // CG state
    SolveLevel& s0 = c->S[0];
    const i64 n = s0.nv * D;
    U.alloc(n, s);
    r.alloc(n, s);
    p.alloc(n, s);
    q.alloc(n, s);
    Fbuf.alloc(n, s);
    Ubuf.alloc(n, s);
    p.zero();
    cg_blocks = (int)std::max<i64>(1, std::min<i64>((i64)sms * 8, ceil_div(n, CG_THREADS)));
    spmv_blocks = (int)std::max<i64>(1, std::min<i64>((i64)sms * 8, ceil_div(s0.nv, CG_THREADS)));
    part.alloc(std::max(cg_blocks, spmv_blocks), s);
    hist.alloc(std::max(1, c->max_iters), s);
    sc.alloc(1, s);
    sc.zero();
    VASMG_CUDA(cudaMallocHost((void**)&host_sc, sizeof(Scalars)));
    cga.nv = (int)s0.nv;
    cga.perm = s0.perm.get();
    cga.isdir = c->isdir.get();
    cga.lift = c->lift.get();
    cga.udir = c->udir.get();
    cga.U = U.get();
    cga.r = r.get();
    cga.p = p.get();
    cga.q = q.get();
    cga.part = part.get();
    cga.hist = hist.get();
    cga.sc = sc.get();
    cga.cond = 0;
    build_sell();
    if (c->gamma >= 2) {
      wb.resize(L);
      we.resize(L);
      for (int l = 1; l < L; ++l) {
        wb[l].alloc(std::max<i64>(1, c->S[l].nv * D), s);
        we[l].alloc(std::max<i64>(1, c->S[l].nv * D), s);
      }
    }
    if (c->autotune) autotune_lanes();
    build_staged_all();
    VASMG_CUDA(cudaStreamSynchronize(s));
  }

  // ---------------------------------------------------------------- staged sweeps (3D)
  // Level l's staged parts for lanes g: each colour step's rows dealt to the
  // NG = STG_T / g groups (longest first, to the group with the fewest slots
  // so far; on the host, from the row pointers), the chunks filled on the device.
  void build_staged(int l, int g) {
    if constexpr (D == 3) {
      cudaStream_t s = c->stream;
      SolveLevel& sl = c->S[l];
      const int nv = (int)sl.nv, C = sl.ncol, R = lv[l].R;
      constexpr int EPT = stg_ept<S>();
      const int NG = STG_T / g;
      VASMG_CHECK(nv < STG_NONE, VASMG_ERR_UNSUPPORTED, "level too large for the staged sweep");
      const std::vector<int> RS = rs_dev[l].download();
      for (int m = 0; m < 2; ++m) {
        Staged& st = stg[m][l];
        if (st.G == g) continue;
        st.G = 0;
        std::vector<int> rp((size_t)nv + 1);
        VASMG_CUDA(cudaMemcpyAsync(rp.data(), m == 0 ? rpl_dev[l].get() : sl.rp.get(), sizeof(int) * (nv + 1),
                                   cudaMemcpyDeviceToHost, s));
        VASMG_CUDA(cudaStreamSynchronize(s));
        std::vector<long long> step_off((size_t)C * R + 1, 0);
        std::vector<int> step_nact((size_t)C * R, 32);
        std::vector<int> goff((size_t)C * R * (NG + 1), 0), srow(std::max(nv, 1), 0);
        std::vector<int> order, load(NG), grp;
        std::vector<std::vector<int>> lists(NG);
        for (int col = 0; col < C; ++col)
          for (int k = 0; k < R; ++k) {
            const size_t step = (size_t)col * R + k;
            const int r0 = RS[(size_t)col * (R + 1) + k], r1 = RS[(size_t)col * (R + 1) + k + 1];
            auto slots = [&](int r) { return std::max(1, (int)ceil_div(rp[r + 1] - rp[r], g)); };
            order.resize(r1 - r0);
            for (int r = r0; r < r1; ++r) order[r - r0] = r;
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return slots(a) > slots(b); });
            std::fill(load.begin(), load.end(), 0);
            for (auto& v : lists) v.clear();
            for (int r : order) {
              const int gi = (int)(std::min_element(load.begin(), load.end()) - load.begin());
              load[gi] += slots(r);
              lists[gi].push_back(r);
            }
            // the groups with rows are 0 .. used-1 (rows go to the first least
            // loaded group); the step's chunks hold their warps only
            int pos = r0, mx = 0, used = 0;
            for (int gi = 0; gi < NG; ++gi) {
              goff[step * (NG + 1) + gi] = pos - r0;
              for (int r : lists[gi]) srow[pos++] = r;
              mx = std::max(mx, load[gi]);
              if (!lists[gi].empty()) used = gi + 1;
            }
            goff[step * (NG + 1) + NG] = pos - r0;
            const int nact = std::min(STG_T, std::max(32, (int)ceil_div(used * g, 32) * 32));
            step_nact[step] = nact;
            step_off[step + 1] = step_off[step] + ceil_div(mx, EPT) * EPT * nact;
          }
        const i64 nslot = step_off[(size_t)C * R];
        st.step_off.alloc((i64)step_off.size(), s);
        st.step_off.upload(step_off.data(), (i64)step_off.size());
        st.step_nact.alloc((i64)step_nact.size(), s);
        st.step_nact.upload(step_nact.data(), (i64)step_nact.size());
        st.goff.alloc((i64)goff.size(), s);
        st.goff.upload(goff.data(), (i64)goff.size());
        st.srow.alloc((i64)srow.size(), s);
        st.srow.upload(srow.data(), (i64)srow.size());
        const i64 ne = std::max<i64>(STG_T * EPT, nslot);
        st.ci.alloc(ne, s);
        st.v8.alloc(ne * 8, s);
        st.v9.alloc(ne, s);
        VASMG_CHECK(((uintptr_t)st.ci.get() | (uintptr_t)st.v8.get() | (uintptr_t)st.v9.get()) % 16 == 0,
                    VASMG_ERR_CUDA, "staged operator not 16-byte aligned");
        st.nslots = nslot;
        st.op.ci = st.ci.get();
        st.op.v8 = st.v8.get();
        st.op.v9 = st.v9.get();
        st.op.step_off = st.step_off.get();
        st.op.step_nact = st.step_nact.get();
        st.op.goff = st.goff.get();
        st.op.srow = st.srow.get();
        st.G = g;
        fill_staged(l, m);
      }
    } else {
      (void)l;
      (void)g;
    }
  }
  // (re)fill level l's staged part m from the level's blocks
  void fill_staged(int l, int m) {
    Staged& st = stg[m][l];
    if (st.G == 0 || st.nslots == 0) return;
    SolveLevel& sl = c->S[l];
    const i64 threads = (i64)sl.ncol * lv[l].R * STG_T;
    if (m == 0)
      stage_fill_kernel<S><<<grid_for(threads, 256), 256, 0, c->stream>>>(
          rpl_dev[l].get(), cil_dev[l].get(), offl_dev[l].get(), nnz_lo[l], lv[l].RS, lv[l].R, sl.ncol,
          st.step_off.get(), st.step_nact.get(), st.goff.get(), st.srow.get(), st.G, st.ci.get(), st.v8.get(),
          st.v9.get());
    else
      stage_fill_kernel<S><<<grid_for(threads, 256), 256, 0, c->stream>>>(
          sl.rp.get(), sl.ci.get(), (const S*)off_ptr(sl), sl.nnz, lv[l].RS, lv[l].R, sl.ncol, st.step_off.get(),
          st.step_nact.get(), st.goff.get(), st.srow.get(), st.G, st.ci.get(), st.v8.get(), st.v9.get());
    check_launch("stage_fill");
  }
  bool staged_on(int l) const {
    return D == 3 && l < lt && stg[0][l].G != 0 && stg[0][l].G == G[l] && stg[1][l].G == G[l];
  }
  template <int GG>
  void occ_staged(int* bd, int* bu) {
    if constexpr (D == 3) {
      VASMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(bd, vstaged_kernel<D, GG, V, S, 0>, STG_T + 32,
                                                               stg_smem_bytes<S>()));
      VASMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(bu, vstaged_kernel<D, GG, V, S, 1>, STG_T + 32,
                                                               stg_smem_bytes<S>()));
    } else {
      *bd = *bu = 0;
    }
  }
  // CTAs of the staged sweeps with g lanes per row that the device holds at once
  i64 staged_capacity(int g) {
    int bd = 0, bu = 0;
    switch (g) {
      case 4: occ_staged<4>(&bd, &bu); break;
      case 8: occ_staged<8>(&bd, &bu); break;
      case 16: occ_staged<16>(&bd, &bu); break;
      default: occ_staged<32>(&bd, &bu); break;
    }
    return (i64)std::min(bd, bu) * sms_;
  }
  template <int GG>
  void staged_attrs() {
    if constexpr (D == 3) {
      VASMG_CUDA(cudaFuncSetAttribute(vstaged_kernel<D, GG, V, S, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      stg_smem_bytes<S>()));
      VASMG_CUDA(cudaFuncSetAttribute(vstaged_kernel<D, GG, V, S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      stg_smem_bytes<S>()));
    }
  }
  // the staged copies of every 3D region level for its lanes G, where the
  // staged kernels can hold the level's region grid
  void build_staged_all() {
    if constexpr (D == 3) {
      for (int l = 0; l < lt; ++l)
        if (staged_capacity(G[l]) >= lv[l].R) build_staged(l, G[l]);
    }
  }

  template <int GG>
  void occ(int* bd, int* bu) {
    VASMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(bd, vdown_kernel<D, GG, V, S>, df_threads<D, V>(), 0));
    VASMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(bu, vup_kernel<D, GG, V, S>, df_threads<D, V>(), 0));
  }
  // CTAs of the sweep kernels with g lanes per row that the device holds at once
  i64 sweep_capacity(int g) {
    int bd = 1, bu = 1;
    switch (g) {
      case 4: occ<4>(&bd, &bu); break;
      case 8: occ<8>(&bd, &bu); break;
      case 16: occ<16>(&bd, &bu); break;
      default: occ<32>(&bd, &bu); break;
    }
    return (i64)std::min(bd, bu) * sms_;
  }

  // For every region level, time the forward sweep, the residual and the
  // backward sweep with each G of {4, 8, 16, 32} whose kernels can hold the
  // level's region grid (CUDA events, one warm-up and three timed runs) and
  // keep the fastest.  A level signature measured before in this process
  // (by this or another handle) reuses that choice.
  void autotune_lanes() {
    cudaStream_t s = c->stream;
    for (int l = 0; l < lt; ++l) {
      const SolveLevel& sl = c->S[l];
      const LaneKey key{D, c->precision, (long long)sl.nv, (long long)sl.nnz};
      {
        std::lock_guard<std::mutex> lock(lane_cache_mutex());
        auto it = lane_cache().find(key);
        if (it != lane_cache().end()) {
          if (sweep_capacity(it->second) >= lv[l].R) G[l] = it->second;
          continue;
        }
      }
      VASMG_CUDA(cudaMemsetAsync(lv[l].x, 0, sizeof(V) * (size_t)sl.nv * D, s));
      VASMG_CUDA(cudaMemsetAsync(lv[l].b, 0, sizeof(V) * (size_t)sl.nv * D, s));
      clear_abort(s);
      cudaEvent_t e0, e1;
      VASMG_CUDA(cudaEventCreate(&e0));
      VASMG_CUDA(cudaEventCreate(&e1));
      int best_g = G[l];
      float best_ms = 0.0f;
      for (int g : {4, 8, 16, 32}) {
        if (sweep_capacity(g) < lv[l].R) continue;
        G[l] = g;
        if (D == 3 && staged_capacity(g) >= lv[l].R) build_staged(l, g);
        auto run = [&]() {
          down(l, 1, s);
          down(l, 2, s);
          up(l, 2, s);
        };
        run();
        VASMG_CUDA(cudaEventRecord(e0, s));
        for (int rep = 0; rep < 3; ++rep) run();
        VASMG_CUDA(cudaEventRecord(e1, s));
        VASMG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        VASMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (best_ms == 0.0f || ms < best_ms) {
          best_ms = ms;
          best_g = g;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      VASMG_CHECK(read_abort(s) == 0, VASMG_ERR_TIMEOUT, "a device wait gave up");
      std::lock_guard<std::mutex> lock(lane_cache_mutex());
      const int chosen = lane_cache().emplace(key, best_g).first->second;  // another handle may have been first
      G[l] = sweep_capacity(chosen) >= lv[l].R ? chosen : best_g;
    }
  }

  // ---------------------------------------------------------------- launches
  // cooperative launch: every CTA (region) of the grid is resident at once
  // cooperative launch of a staged sweep (producer warp, shared-memory ring)
  template <typename K>
  void launch_coop_staged(K kern, int grid, const LV<V>& a, const StagedOp<S>& o, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(STG_T + 32);
    cfg.dynamicSmemBytes = stg_smem_bytes<S>();
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    Scalars* scp = sc.get();
    VASMG_CUDA(cudaLaunchKernelEx(&cfg, kern, a, o, scp));
    ++launch_counter;
  }
  template <int MODE>
  void sweep_staged(int l, cudaStream_t s) {
    if constexpr (D == 3) {
      const StagedOp<S>& o = stg[MODE][l].op;
      const int g = lv[l].R;
      switch (G[l]) {
        case 4: launch_coop_staged(vstaged_kernel<D, 4, V, S, MODE>, g, lv[l], o, s); break;
        case 8: launch_coop_staged(vstaged_kernel<D, 8, V, S, MODE>, g, lv[l], o, s); break;
        case 16: launch_coop_staged(vstaged_kernel<D, 16, V, S, MODE>, g, lv[l], o, s); break;
        default: launch_coop_staged(vstaged_kernel<D, 32, V, S, MODE>, g, lv[l], o, s); break;
      }
    } else {
      (void)l;
      (void)s;
    }
  }
  template <typename K>
  void launch_coop(K kern, int grid, const LV<V>& a, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(df_threads<D, V>());
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    Scalars* scp = sc.get();
    VASMG_CUDA(cudaLaunchKernelEx(&cfg, kern, a, scp));
    ++launch_counter;
  }
  int plain_grid(i64 threads) const { return (int)std::max<i64>(1, std::min<i64>(ceil_div(threads, 256), sms_ * 8)); }
  template <int GG>
  void residual(int l, cudaStream_t s) {
    residual_kernel<D, GG, V, S><<<plain_grid((i64)lv[l].nv * GG), 256, 0, s>>>(lv[l]);
    ++launch_counter;
  }
  // phases: 1 forward sweep (zero start), 2 residual, 4 restriction
  void down(int l, int phases, cudaStream_t s) {
    const int g = lv[l].R;
    if ((phases & 1) && staged_on(l)) {
      sweep_staged<0>(l, s);
    } else if (phases & 1) {
      switch (G[l]) {
        case 4: launch_coop(vdown_kernel<D, 4, V, S>, g, lv[l], s); break;
        case 8: launch_coop(vdown_kernel<D, 8, V, S>, g, lv[l], s); break;
        case 16: launch_coop(vdown_kernel<D, 16, V, S>, g, lv[l], s); break;
        default: launch_coop(vdown_kernel<D, 32, V, S>, g, lv[l], s); break;
      }
    }
    if (phases & 2) {
      switch (G[l]) {
        case 4: residual<4>(l, s); break;
        case 8: residual<8>(l, s); break;
        case 16: residual<16>(l, s); break;
        default: residual<32>(l, s); break;
      }
    }
    if (phases & 4) {
      restrict_kernel<D, V><<<plain_grid(lv[l].nvc), 256, 0, s>>>(lv[l]);
      ++launch_counter;
    }
  }
  // phases: 1 prolongation + correction, 2 backward sweep
  void up(int l, int phases, cudaStream_t s) {
    if (phases & 1) {
      prolong_kernel<D, V><<<plain_grid(lv[l].nv), 256, 0, s>>>(lv[l]);
      ++launch_counter;
    }
    if ((phases & 2) && staged_on(l)) {
      sweep_staged<1>(l, s);
    } else if (phases & 2) {
      const int g = lv[l].R;
      switch (G[l]) {
        case 4: launch_coop(vup_kernel<D, 4, V, S>, g, lv[l], s); break;
        case 8: launch_coop(vup_kernel<D, 8, V, S>, g, lv[l], s); break;
        case 16: launch_coop(vup_kernel<D, 16, V, S>, g, lv[l], s); break;
        default: launch_coop(vup_kernel<D, 32, V, S>, g, lv[l], s); break;
      }
    }
  }
  // First level of the one-CTA part of a tail that starts at level l0.
  int one_cta_start(int l0) const {
    int ls = L - 1;
    while (ls > l0 && c->S[ls - 1].nv <= ONE_CTA_NV) --ls;
    return ls;
  }
  // The tail's level tables; levels ls..L-1 get shared-memory slots.
  // Returns the dynamic shared memory in bytes.
  size_t fill_tail_args(TailArgs<V>& ta, int l0, int ls) {
    std::memset(&ta, 0, sizeof(ta));
    ta.l0 = l0;
    ta.L = L - 1;
    ta.ls = ls;
    ta.kd = -1;
    size_t smem = 0;
    for (int l = ta.ls; l < L; ++l) {
      ta.soff[l] = (int)(smem / sizeof(V));
      smem += 3 * sizeof(V) * (size_t)c->S[l].nv * D;
      smem = (smem + 15) / 16 * 16;
    }
    VASMG_CHECK(smem <= (size_t)TAIL_SMEM_MAX, VASMG_ERR_UNSUPPORTED, "tail levels too large for shared memory");
    for (int l = 0; l < L; ++l) {
      const LV<V>& v = lv[l];
      TL<V>& t = ta.lv[l];
      t.nv = v.nv;
      t.nnz = v.nnz;
      t.rp = v.rp;
      t.ci = v.ci;
      t.sp = v.sp;
      t.off = v.off;
      t.dinv = v.dinv;
      t.dead = v.dead;
      t.x = v.x;
      t.b = v.b;
      t.r = v.r;
      t.cs = v.cs;
      t.ncol = v.ncol;
      t.nvc = v.nvc;
      t.prp = v.prp;
      t.pci = v.pci;
      t.pw = v.pw;
      t.rrp = v.rrp;
      t.rci = v.rci;
      t.rw = v.rw;
      t.bc = v.bc;
      t.xc = v.xc;
    }
    ta.co = co;
    return smem;
  }
  // The V-cycle from the dense level kd down, as the matrix M (one CTA per
  // column, the same arithmetic as the tail's one-CTA part).  Rebuilt when
  // the operators' values change.
  void dense_level(int* k, int* n) const override {
    *k = kd;
    *n = dn;
  }
  void lanes(int32_t* g, int n) const override {
    for (int l = 0; l < n; ++l) g[l] = l < lt && l < (int)G.size() ? G[l] : 0;
  }
  void staged(int l, int64_t* v) const override {
    for (int q = 0; q < 5; ++q) v[q] = 0;
    if (l < 0 || l >= L || !staged_on(l)) return;
    v[0] = stg[0][l].nslots;
    v[1] = nnz_lo[l];
    v[2] = stg[1][l].nslots;
    v[3] = c->S[l].nnz;
    v[4] = 4 + 9 * (i64)sizeof(S);
  }
  void build_dense_level() {
    kd = -1;
    dn = 0;
    // the dense matrix is the V-cycle below its level; gamma >= 2 runs every
    // level with per-level launches instead
    if (!c->dense_coarse || c->gamma >= 2) return;
    if constexpr (std::is_same<V, float>::value) {
      const int ls = one_cta_start(lt);
      for (int l = ls; l < L; ++l) {
        const i64 n = c->S[l].nv * D;
        if (n * n <= (i64)nct * DENSE_ROWS_PER_CTA * DENSE_ROWS_PER_CTA) {
          kd = l;
          break;
        }
      }
      if (kd < 0) return;
      cudaStream_t s = c->stream;
      dn = (int)(c->S[kd].nv * D);
      dld = (dn + 3) / 4 * 4;
      {
        // the tail stages b_kd in shared memory beside its levels' vectors
        TailArgs<V> probe;
        const size_t need = fill_tail_args(probe, lt, ls) + sizeof(V) * (size_t)dld;
        if (need > (size_t)TAIL_SMEM_MAX) {
          kd = -1;
          dn = 0;
          return;
        }
      }
      if (dm.n != (i64)dn * dld) dm.alloc((i64)dn * dld, s);
      dm.zero();
      DevBuf<double> ys;
      ys.alloc((i64)dn * co.n, s);
      TailArgs<V> ta;
      const size_t smem = fill_tail_args(ta, kd, kd);
      ta.dn = dn;
      ta.dld = dld;
      dense_level_kernel<D, V, S><<<dn, TAIL_THREADS, smem, s>>>(ta, dm.get(), ys.get());
      check_launch("dense_level");
    }
  }
  void tail(int l0, cudaStream_t s) {
    TailArgs<V> ta;
    size_t smem = fill_tail_args(ta, l0, one_cta_start(l0));
    if (kd >= 0 && kd >= ta.ls) {
      ta.kd = kd;
      ta.dn = dn;
      ta.dld = dld;
      ta.dm = dm.get();
      ta.dsoff = (int)(smem / sizeof(V));  // fill_tail_args keeps smem a multiple of 16 bytes
      smem += sizeof(V) * (size_t)dld;
      VASMG_CHECK(smem <= (size_t)TAIL_SMEM_MAX, VASMG_ERR_UNSUPPORTED, "tail levels too large for shared memory");
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nct);
    cfg.blockDim = dim3(TAIL_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nct;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    VASMG_CUDA(cudaLaunchKernelEx(&cfg, tail_kernel<D, V, S>, ta));
    ++launch_counter;
  }
  // V-cycle from level l0 (b_{l0} set, result in x_{l0}).
  void vcycle(int l0, cudaStream_t s) {
    if (l0 >= lt) {
      tail(l0, s);
      return;
    }
    for (int l = l0; l < lt; ++l) down(l, 7, s);
    tail(lt, s);
    for (int l = lt - 1; l >= l0; --l) up(l, 3, s);
  }

  void vec_copy(V* dst, const V* src, i64 n, cudaStream_t s) {
    vcopy_kernel<V><<<plain_grid(n), 256, 0, s>>>(dst, src, n);
    ++launch_counter;
  }
  void vec_add(V* dst, const V* src, i64 n, cudaStream_t s) {
    vadd_kernel<V><<<plain_grid(n), 256, 0, s>>>(dst, src, n);
    ++launch_counter;
  }
  // b_l = bs - A_l x_l
  void full_residual(int l, const V* bs, cudaStream_t s) {
    const double* dg = c->S[l].diag64.get();
    const int grid = plain_grid((i64)lv[l].nv * G[l]);
    switch (G[l]) {
      case 4: full_residual_kernel<D, 4, V, S><<<grid, 256, 0, s>>>(lv[l], dg, bs, lv[l].b); break;
      case 8: full_residual_kernel<D, 8, V, S><<<grid, 256, 0, s>>>(lv[l], dg, bs, lv[l].b); break;
      case 16: full_residual_kernel<D, 16, V, S><<<grid, 256, 0, s>>>(lv[l], dg, bs, lv[l].b); break;
      default: full_residual_kernel<D, 32, V, S><<<grid, 256, 0, s>>>(lv[l], dg, bs, lv[l].b); break;
    }
    ++launch_counter;
  }
  // The cycle with gamma coarse corrections from level l (b_l set, result in
  // x_l), one launch per step and level: zero start, forward sweep, residual,
  // restriction; the coarse problem by gamma cycles, each after the first on
  // the updated coarse residual (one only when the coarser level is the
  // coarsest, which is solved directly); prolongation, backward sweep.
  void gcycle(int l, cudaStream_t s) {
    if (l == L - 1) {
      coarse_kernel<V><<<1, 32, 0, s>>>(co, lv[L - 1].b, lv[L - 1].x);
      ++launch_counter;
      return;
    }
    down(l, 7, s);
    gcycle(l + 1, s);
    const int reps = l + 2 == L ? 1 : c->gamma;
    if (reps > 1) {
      const i64 nc = (i64)lv[l + 1].nv * D;
      vec_copy(wb[l + 1].get(), lv[l + 1].b, nc, s);
      for (int rep = 1; rep < reps; ++rep) {
        vec_copy(we[l + 1].get(), lv[l + 1].x, nc, s);
        full_residual(l + 1, wb[l + 1].get(), s);
        gcycle(l + 1, s);
        vec_add(lv[l + 1].x, we[l + 1].get(), nc, s);
      }
    }
    up(l, 3, s);
  }
  void cycle_from(int l, cudaStream_t s) {
    if (c->gamma >= 2) gcycle(l, s);
    else vcycle(l, s);
  }
  // The preconditioner: the cycle from level 0, or the additive form of
  // Sec. 4, x_0 = S b_0 + P B_1 R b_0 (S: forward then backward sweep from
  // zero; B_1: the cycle from level 1).
  void precond(cudaStream_t s) {
    if (!c->additive || L == 1) {
      cycle_from(0, s);
      return;
    }
    vec_copy(lv[0].r, lv[0].b, (i64)lv[0].nv * D, s);
    down(0, 4, s);   // b_1 = R b_0
    cycle_from(1, s);
    down(0, 1, s);   // x_0 = forward sweep from zero
    up(0, 2, s);     // backward sweep
    up(0, 1, s);     // x_0 += P x_1
  }

  void spmv(cudaStream_t s, int with_dot) {
    if (cga.cond)
      spmv_sell_kernel<D, true><<<spmv_blocks, CG_THREADS, 0, s>>>(cga, with_dot);
    else
      spmv_sell_kernel<D, false><<<spmv_blocks, CG_THREADS, 0, s>>>(cga, with_dot);
    ++launch_counter;
  }

  // One PCG iteration, rotated so the stop test ends it: z = M r; rho, beta;
  // p = z + beta p; q = A p, alpha; U, r update + stop test.
  void body(cudaStream_t s) {
    V* z = lv[0].x;
    precond(s);
    if (cga.cond)
      rz_kernel<D, V, true><<<cg_blocks, CG_THREADS, 0, s>>>(cga, z);
    else
      rz_kernel<D, V, false><<<cg_blocks, CG_THREADS, 0, s>>>(cga, z);
    p_update_kernel<D, V><<<cg_blocks, CG_THREADS, 0, s>>>(cga, z);
    spmv(s, 1);
    if (cga.cond)
      cg_update_kernel<D, V, true><<<cg_blocks, CG_THREADS, 0, s>>>(cga, lv[0].b);
    else
      cg_update_kernel<D, V, false><<<cg_blocks, CG_THREADS, 0, s>>>(cga, lv[0].b);
    launch_counter += 3;
  }

  // The whole solve as one graph: init -> WHILE(not converged){ body } -> final.
  bool build_while_graph() {
    cudaStream_t s = c->stream;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
    bool ok = true;
    cudaGraphConditionalHandle h = 0;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) ok = false;
    cudaGraph_t out = nullptr;
    cudaGraphNode_t init_node = nullptr, wnode = nullptr;
    if (ok) {
      cga.cond = (unsigned long long)h;
      ok = cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        cg_init_kernel<D, V, true><<<cg_blocks, CG_THREADS, 0, s>>>(cga, Fbuf.get(), lv[0].b);
        ok = cudaStreamEndCapture(s, &out) == cudaSuccess;
      }
    }
    if (ok) {
      size_t nn = 0;
      ok = cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn == 1;
      if (ok) ok = cudaGraphGetNodes(g, &init_node, &nn) == cudaSuccess;
    }
    if (ok) {
      cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      ok = cudaGraphAddNode(&wnode, g, &init_node, nullptr, 1, &np) == cudaSuccess;
      if (ok) {
        cudaGraph_t bodyg = np.conditional.phGraph_out[0];
        launch_counter = 0;
        ok = cudaStreamBeginCaptureToGraph(s, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
          try {
            body(s);
          } catch (...) {
            ok = false;
          }
          ok = (cudaStreamEndCapture(s, &out) == cudaSuccess) && ok;
        }
        launches_body = launch_counter;
      }
    }
    if (ok) {
      ok = cudaStreamBeginCaptureToGraph(s, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        cg_final_kernel<D><<<cg_blocks, CG_THREADS, 0, s>>>(cga, Ubuf.get());
        ok = cudaStreamEndCapture(s, &out) == cudaSuccess;
      }
    }
    if (ok && cudaGraphInstantiate(&exec_while, g, 0) != cudaSuccess) {
      exec_while = nullptr;
      ok = false;
    }
    cudaGraphDestroy(g);
    cudaGetLastError();
    if (!ok) cga.cond = 0;
    return ok;
  }

  void build_graphs() {
    cudaStream_t s = c->stream;
    if (c->use_graph && build_while_graph()) return;
    // per-iteration graph; the host loop reads the stop flag after each iteration
    cga.cond = 0;
    cudaGraph_t bg = nullptr;
    launch_counter = 0;
    VASMG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
      body(s);
    } catch (...) {
      // leave the stream out of capture mode before reporting the error
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(s, &junk);
      if (junk) cudaGraphDestroy(junk);
      cudaGetLastError();
      throw;
    }
    VASMG_CUDA(cudaStreamEndCapture(s, &bg));
    launches_body = launch_counter;
    VASMG_CUDA(cudaGraphInstantiate(&exec_body, bg, 0));
    cudaGraphDestroy(bg);
  }

  int solve(Ctx& ctx, const double* F, double* Uout, double tol, vasmg_stats* st) override {
    cudaStream_t s = c->stream;
    if (!exec_while && !exec_body) build_graphs();
    const i64 n = c->n;
    Scalars init{};
    init.tol = tol;
    init.max_iters = c->max_iters;
    VASMG_CUDA(cudaMemcpyAsync(sc.get(), &init, sizeof(Scalars), cudaMemcpyHostToDevice, s));
    VASMG_CUDA(cudaMemcpyAsync(Fbuf.get(), F, sizeof(double) * n, cudaMemcpyDefault, s));
    if (exec_while) {
      VASMG_CUDA(cudaGraphLaunch(exec_while, s));
      VASMG_CUDA(cudaMemcpyAsync(host_sc, sc.get(), sizeof(Scalars), cudaMemcpyDeviceToHost, s));
      VASMG_CUDA(cudaStreamSynchronize(s));
    } else {
      cg_init_kernel<D, V, false><<<cg_blocks, CG_THREADS, 0, s>>>(cga, Fbuf.get(), lv[0].b);
      check_launch("cg_init");
      VASMG_CUDA(cudaMemcpyAsync(host_sc, sc.get(), sizeof(Scalars), cudaMemcpyDeviceToHost, s));
      VASMG_CUDA(cudaStreamSynchronize(s));
      int guard = 0;
      while (!host_sc->done && guard++ <= c->max_iters) {
        VASMG_CUDA(cudaGraphLaunch(exec_body, s));
        VASMG_CUDA(cudaMemcpyAsync(host_sc, sc.get(), sizeof(Scalars), cudaMemcpyDeviceToHost, s));
        VASMG_CUDA(cudaStreamSynchronize(s));
      }
      cg_final_kernel<D><<<cg_blocks, CG_THREADS, 0, s>>>(cga, Ubuf.get());
      check_launch("cg_final");
    }
    VASMG_CUDA(cudaMemcpyAsync(Uout, Ubuf.get(), sizeof(double) * n, cudaMemcpyDefault, s));
    VASMG_CUDA(cudaStreamSynchronize(s));
    const int iters = host_sc->iter;
    ctx.last_launches = 2 + launches_body * (i64)iters;
    if (st) {
      st->iterations = iters;
      st->rel_res = host_sc->relres;
      st->n_levels = L;
      if (st->res_history && st->res_history_cap > 0) {
        const int k = std::min(st->res_history_cap, std::min(iters, c->max_iters));
        if (k > 0) VASMG_CUDA(cudaMemcpy(st->res_history, hist.get(), sizeof(double) * k, cudaMemcpyDeviceToHost));
      }
    }
    if (host_sc->abort) return VASMG_ERR_TIMEOUT;
    return host_sc->status;
  }

  // ---------------------------------------------------------------- several right-hand sides
  EngineView<V> view() {
    EngineView<V> v;
    v.stream = c->stream;
    v.L = L;
    v.lt = lt;
    v.nct = nct;
    v.sms = sms_;
    v.max_iters = c->max_iters;
    v.use_graph = c->use_graph;
    v.lv = lv;
    v.G = G;
    for (int l = 0; l < L; ++l) {
      v.nv.push_back(c->S[l].nv);
      v.pnnz.push_back(l + 1 < L ? (double)c->C[l].pnnz : 0.0);
    }
    v.tail_smem = fill_tail_args(v.ta, lt, one_cta_start(lt));
    if (kd >= 0 && kd >= v.ta.ls) {
      v.ta.kd = kd;
      v.ta.dn = dn;
      v.ta.dld = dld;
      v.ta.dm = dm.get();
      v.ta.dsoff = (int)(v.tail_smem / sizeof(V));
    }
    v.cga = cga;
    v.cga.cond = 0;
    v.cg_blocks = cg_blocks;
    v.spmv_blocks = spmv_blocks;
    v.sell_real_entries = sell_real_entries;
    v.ctr = ctrs.get();
    v.dim = D;
    v.device = c->device;
    v.Fbuf = Fbuf.get();
    v.Ubuf = Ubuf.get();
    for (int l = 0; l < L; ++l) {
      const bool on = staged_on(l);
      v.stg_fwd.push_back(on ? (const void*)&stg[0][l].op : nullptr);
      v.stg_bwd.push_back(on ? (const void*)&stg[1][l].op : nullptr);
    }
    return v;
  }
  MultiBase* get_multi() {
    if constexpr (std::is_same<V, float>::value) {
      if (!multi) multi = make_multi<D, S>(view());
      else multi->set_view(view());
      return multi;
    }
    return nullptr;
  }
  int solve_multi(Ctx& ctx, int k, const double* const* F, double* const* Uo, double tol, vasmg_stats* st) override {
    if (k == 1) return solve(ctx, F[0], Uo[0], tol, st);
    const bool variant = c->gamma != 1 || c->additive;
    if constexpr (std::is_same<V, float>::value) {
      if (!variant) {
        i64 launches = 0;
        const int rc = get_multi()->solve(k, F, Uo, tol, st, &launches);
        ctx.last_launches = launches;
        return rc;
      }
    }
    {
      // the FP64 V-cycle and the cycle variants: one solve after another
      int worst = VASMG_OK;
      i64 launches = 0;
      for (int i = 0; i < k; ++i) {
        const int rc = solve(ctx, F[i], Uo[i], tol, st ? st + i : nullptr);
        launches += ctx.last_launches;
        if (rc < 0) worst = std::min(worst, rc);
        else if (worst >= 0) worst = std::max(worst, rc);
      }
      ctx.last_launches = launches;
      return worst;
    }
  }
  bool batch_view(EngineView<float>* out) override {
    if constexpr (std::is_same<V, float>::value) {
      if (c->gamma != 1 || c->additive) return false;
      *out = view();
      return true;
    }
    (void)out;
    return false;
  }
  int storage() const override {
    return std::is_same<S, double>::value ? 0 : (std::is_same<S, float>::value ? 1 : 2);
  }
  double time_multi(Ctx& ctx, int which, int level, int k, int reps, double* bytes) override {
    (void)ctx;
    if constexpr (std::is_same<V, float>::value) {
      return get_multi()->time(which, level, k, reps, bytes);
    } else {
      throw Error(VASMG_ERR_UNSUPPORTED, "several right-hand sides per launch need an FP32-vector V-cycle");
    }
  }

  // ---------------------------------------------------------------- single steps
  void to_solve(const double* x, V* out, int l, cudaStream_t s) {
    to_solve_kernel<V><<<grid_for((i64)lv[l].nv * D, 256), 256, 0, s>>>(x, out, c->S[l].perm.get(), lv[l].nv, D);
  }
  void from_solve(const V* in, double* y, int l, cudaStream_t s) {
    from_solve_kernel<V><<<grid_for((i64)lv[l].nv * D, 256), 256, 0, s>>>(in, y, c->S[l].perm.get(), lv[l].nv, D);
  }
  void clear_abort(cudaStream_t s) { VASMG_CUDA(cudaMemsetAsync(&sc.get()->abort, 0, sizeof(int), s)); }
  int read_abort(cudaStream_t s) {
    int a = 0;
    VASMG_CUDA(cudaMemcpyAsync(&a, &sc.get()->abort, sizeof(int), cudaMemcpyDeviceToHost, s));
    VASMG_CUDA(cudaStreamSynchronize(s));
    return a;
  }

  void apply(Ctx& ctx, int op, int l, const double* x, double* y) override {
    cudaStream_t s = c->stream;
    VASMG_CHECK(l >= 0 && l < L, VASMG_ERR_INVALID_ARG, "level out of range");
    const bool has_coarser = l + 1 < L;
    clear_abort(s);
    switch (op) {
      case VASMG_OP_MATVEC: {
        VASMG_CHECK(l == 0, VASMG_ERR_INVALID_ARG, "MATVEC runs the level-0 FP64 operator");
        to_solve_kernel<double><<<grid_for((i64)lv[0].nv * D, 256), 256, 0, s>>>(x, p.get(), c->S[0].perm.get(),
                                                                                    lv[0].nv, D);
        spmv(s, 0);
        from_solve_kernel<double><<<grid_for((i64)lv[0].nv * D, 256), 256, 0, s>>>(q.get(), y, c->S[0].perm.get(),
                                                                                      lv[0].nv, D);
        p.zero();
        break;
      }
      case VASMG_OP_SMOOTH_FWD:
        VASMG_CHECK(has_coarser, VASMG_ERR_INVALID_ARG, "the coarsest level is solved directly");
        to_solve(x, lv[l].b, l, s);
        down(l, 1, s);
        from_solve(lv[l].x, y, l, s);
        break;
      case VASMG_OP_SMOOTH_BWD:
        VASMG_CHECK(has_coarser, VASMG_ERR_INVALID_ARG, "the coarsest level is solved directly");
        to_solve(x, lv[l].b, l, s);
        to_solve(y, lv[l].x, l, s);
        up(l, 2, s);
        from_solve(lv[l].x, y, l, s);
        break;
      case VASMG_OP_RESIDUAL:
        VASMG_CHECK(has_coarser, VASMG_ERR_INVALID_ARG, "the coarsest level is solved directly");
        to_solve(x, lv[l].b, l, s);
        down(l, 3, s);
        from_solve(lv[l].r, y, l, s);
        break;
      case VASMG_OP_RESTRICT:
        VASMG_CHECK(has_coarser, VASMG_ERR_INVALID_ARG, "no coarser level");
        to_solve(x, lv[l].r, l, s);
        down(l, 4, s);
        from_solve(lv[l + 1].b, y, l + 1, s);
        break;
      case VASMG_OP_PROLONG:
        VASMG_CHECK(has_coarser, VASMG_ERR_INVALID_ARG, "no coarser level");
        to_solve(x, lv[l + 1].x, l + 1, s);
        to_solve(y, lv[l].x, l, s);
        up(l, 1, s);
        from_solve(lv[l].x, y, l, s);
        break;
      case VASMG_OP_COARSE:
        to_solve(x, lv[L - 1].b, L - 1, s);
        coarse_kernel<V><<<1, 32, 0, s>>>(co, lv[L - 1].b, lv[L - 1].x);
        from_solve(lv[L - 1].x, y, L - 1, s);
        break;
      case VASMG_OP_VCYCLE:
        to_solve(x, lv[l].b, l, s);
        cycle_from(l, s);
        from_solve(lv[l].x, y, l, s);
        break;
      case VASMG_OP_PRECOND:
        VASMG_CHECK(l == 0, VASMG_ERR_INVALID_ARG, "the preconditioner acts on level 0");
        to_solve(x, lv[0].b, 0, s);
        precond(s);
        from_solve(lv[0].x, y, 0, s);
        break;
      default:
        throw Error(VASMG_ERR_INVALID_ARG, "unknown op");
    }
    check_launch("apply");
    VASMG_CUDA(cudaStreamSynchronize(s));
    VASMG_CHECK(read_abort(s) == 0, VASMG_ERR_TIMEOUT, "a device wait gave up");
    (void)ctx;
  }

  // ---------------------------------------------------------------- timing
  // Algorithmic bytes: every array the step must touch, each element once.
  double pass_bytes(int l) {  // one pass over the off-diagonal blocks + row pointers
    const SolveLevel& sl = c->S[l];
    return (double)sl.nnz * (D * D * sizeof(S) + 4.0) + (sl.nv + 1.0) * 4.0 + (double)sl.nv * 4.0;
  }
  double down_bytes(int l) {
    const SolveLevel& sl = c->S[l];
    const double n = (double)sl.nv * D;
    double b = pass_bytes(l) + (double)sl.nv * D * D * sizeof(V) + 4.0 * n * sizeof(V);  // b, x w+r, r w
    if (l + 1 < L) {
      const double pn = (double)c->C[l].pnnz;
      b += n * sizeof(V) + pn * (4.0 + sizeof(V)) + (c->S[l + 1].nv + 1.0) * 4.0 +
           (double)c->S[l + 1].nv * D * sizeof(V);
    }
    return b;
  }
  double sweep_bytes(int l) {
    const SolveLevel& sl = c->S[l];
    const double n = (double)sl.nv * D;
    return pass_bytes(l) + (double)sl.nv * D * D * sizeof(V) + 3.0 * n * sizeof(V);  // b, x r+w
  }
  double up_bytes(int l) {
    double b = sweep_bytes(l);
    if (l + 1 < L) {
      const double pn = (double)c->C[l].pnnz;
      b += pn * (4.0 + sizeof(V)) + (c->S[l].nv + 1.0) * 4.0 + (double)c->S[l].nv +
           (double)c->S[l + 1].nv * D * sizeof(V) + 2.0 * (double)c->S[l].nv * D * sizeof(V);
    }
    return b;
  }
  // single kernels (each array the kernel must touch, each element once)
  double fwd_bytes(int l) {  // lower blocks, rp/sp, dinv, b read, x written (and gathered)
    const SolveLevel& sl = c->S[l];
    const double n = (double)sl.nv * D;
    return (double)nnz_lo[l] * (D * D * sizeof(S) + 4.0) + 8.0 * sl.nv + (double)sl.nv * D * D * sizeof(V) +
           3.0 * n * sizeof(V);
  }
  double residual_bytes(int l) {  // upper blocks, sp/rp, x read, r written
    const SolveLevel& sl = c->S[l];
    const double n = (double)sl.nv * D;
    return (double)(sl.nnz - nnz_lo[l]) * (D * D * sizeof(S) + 4.0) + 8.0 * sl.nv + 2.0 * n * sizeof(V);
  }
  double restrict_bytes(int l) {  // R entries, row pointers, r read, b_{l+1} written
    const double pn = (double)c->C[l].pnnz;
    return pn * (4.0 + sizeof(V)) + (c->S[l + 1].nv + 1.0) * 4.0 + (double)c->S[l].nv * D * sizeof(V) +
           (double)c->S[l + 1].nv * D * sizeof(V);
  }
  double prolong_bytes(int l) {  // P entries, row pointers, dead bits, x_{l+1} read, x_l read + written
    const double pn = (double)c->C[l].pnnz;
    return pn * (4.0 + sizeof(V)) + (c->S[l].nv + 1.0) * 4.0 + (double)c->S[l].nv +
           (double)c->S[l + 1].nv * D * sizeof(V) + 2.0 * (double)c->S[l].nv * D * sizeof(V);
  }
  double tail_bytes(int l0) {
    if (kd >= 0 && kd >= one_cta_start(l0)) {
      // levels l0..kd-1, then M (with its padding) and b_kd, x_kd
      double b = (double)dn * dld * sizeof(V) + 2.0 * dn * sizeof(V);
      for (int l = l0; l < kd; ++l) b += down_bytes(l) + up_bytes(l);
      return b;
    }
    double b = (double)c->nc * c->nc * 8.0;
    for (int l = l0; l + 1 < L; ++l) b += down_bytes(l) + up_bytes(l);
    return b;
  }
  double spmv_bytes() {
    const SolveLevel& sl = c->S[0];
    const double n = (double)sl.nv * D;
    return (double)sell_real_entries * (D * D * 8.0 + 4.0) + 3.0 * n * 8.0;  // blocks, p read, q write, p for the dot
  }
  double vcycle_bytes() {
    double b = 0;
    for (int l = 0; l + 1 < L; ++l) b += down_bytes(l) + up_bytes(l);
    return b;
  }

  double time(Ctx& ctx, int which, int level, int reps, double* bytes) override {
    cudaStream_t s = c->stream;
    VASMG_CHECK(which >= VASMG_KERNEL_SPMV64 && which <= VASMG_KERNEL_TAIL, VASMG_ERR_INVALID_ARG, "unknown kernel");
    VASMG_CHECK(which != VASMG_KERNEL_TAIL || level >= lt, VASMG_ERR_INVALID_ARG, "level is not in the tail launch");
    VASMG_CHECK(which == VASMG_KERNEL_SPMV64 || which == VASMG_KERNEL_VCYCLE || level + 1 < L, VASMG_ERR_INVALID_ARG,
                "the coarsest level has no sweep");
    clear_abort(s);
    cudaEvent_t e0, e1;
    VASMG_CUDA(cudaEventCreate(&e0));
    VASMG_CUDA(cudaEventCreate(&e1));
    auto run = [&]() {
      switch (which) {
        case VASMG_KERNEL_SPMV64: spmv(s, 0); break;
        case VASMG_KERNEL_SWEEP: up(level, 2, s); break;
        case VASMG_KERNEL_DOWN: down(level, 7, s); break;
        case VASMG_KERNEL_UP: up(level, 3, s); break;
        case VASMG_KERNEL_FWD_SWEEP: down(level, 1, s); break;
        case VASMG_KERNEL_RESIDUAL: down(level, 2, s); break;
        case VASMG_KERNEL_RESTRICT: down(level, 4, s); break;
        case VASMG_KERNEL_PROLONG: up(level, 1, s); break;
        case VASMG_KERNEL_TAIL: tail(level, s); break;
        default: vcycle(0, s); break;
      }
    };
    run();
    VASMG_CUDA(cudaStreamSynchronize(s));
    VASMG_CUDA(cudaEventRecord(e0, s));
    for (int i = 0; i < reps; ++i) run();
    VASMG_CUDA(cudaEventRecord(e1, s));
    VASMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    VASMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    VASMG_CHECK(read_abort(s) == 0, VASMG_ERR_TIMEOUT, "a device wait gave up");
    switch (which) {
      case VASMG_KERNEL_SPMV64: *bytes = spmv_bytes(); break;
      case VASMG_KERNEL_SWEEP: *bytes = sweep_bytes(level); break;
      case VASMG_KERNEL_DOWN: *bytes = down_bytes(level); break;
      case VASMG_KERNEL_UP: *bytes = up_bytes(level); break;
      case VASMG_KERNEL_FWD_SWEEP: *bytes = fwd_bytes(level); break;
      case VASMG_KERNEL_RESIDUAL: *bytes = residual_bytes(level); break;
      case VASMG_KERNEL_RESTRICT: *bytes = restrict_bytes(level); break;
      case VASMG_KERNEL_PROLONG: *bytes = prolong_bytes(level); break;
      case VASMG_KERNEL_TAIL: *bytes = tail_bytes(level); break;
      default: *bytes = vcycle_bytes(); break;
    }
    (void)ctx;
    return (double)ms / reps;
  }
};

void setup_solver_state(Ctx& c) {
  if (c.dim == 2) {
    if (c.precision == VASMG_FP64) c.eng = new Engine<2, double, double>(c);
    else if (c.precision == VASMG_FP32_VCYCLE) c.eng = new Engine<2, float, float>(c);
    else c.eng = new Engine<2, float, __nv_bfloat16>(c);
  } else {
    if (c.precision == VASMG_FP64) c.eng = new Engine<3, double, double>(c);
    else if (c.precision == VASMG_FP32_VCYCLE) c.eng = new Engine<3, float, float>(c);
    else c.eng = new Engine<3, float, __nv_bfloat16>(c);
  }
}

void refresh_solver_values(Ctx& c) { c.eng->refresh_values(); }

void destroy_solver_state(Ctx& c) {
  delete c.eng;
  c.eng = nullptr;
}

int solve_dev(Ctx& c, const double* F_dev, double* U_dev, double tol, vasmg_stats* st) {
  return c.eng->solve(c, F_dev, U_dev, tol, st);
}

void apply_op(Ctx& c, int op, int level, const double* x_dev, double* y_dev) {
  c.eng->apply(c, op, level, x_dev, y_dev);
}

double time_kernel(Ctx& c, int which, int level, int reps, double* bytes) {
  return c.eng->time(c, which, level, reps, bytes);
}

int solve_multi_dev(Ctx& c, int k, const double* const* F, double* const* U, double tol, vasmg_stats* st) {
  return c.eng->solve_multi(c, k, F, U, tol, st);
}

// The batched launch of vasmg_solve_batch, or -1000 if these handles cannot
// share launches (the caller then overlaps single solves): all with FP32
// vectors, one storage precision, the plain V-cycle, the current device.
// Handles whose regions do not fit the device together run in successive
// groups, each one launch per level and phase.
int solve_batch_dev(const std::vector<Ctx*>& cs, const double* const* F, double* const* U, double tol,
                    vasmg_stats* st, i64* launches) {
  const int k = (int)cs.size();
  if (k < 2) return -1000;
  int dev = 0;
  VASMG_CUDA(cudaGetDevice(&dev));
  const int sto = cs[0]->eng->storage();
  std::vector<EngineView<float>> views(k);
  for (int i = 0; i < k; ++i) {
    if (cs[i]->device != dev || cs[i]->eng->storage() != sto || !cs[i]->eng->batch_view(&views[i])) return -1000;
    for (int j = 0; j < i; ++j)
      if (cs[j] == cs[i]) return -1000;
  }
  const int cap = sto == 1 ? batch_sweep_capacity<float>() : batch_sweep_capacity<__nv_bfloat16>();
  for (const auto& v : views)
    for (int l = 0; l < v.lt; ++l)
      if (v.lv[l].R > cap) return -1000;
  // every handle's earlier work first
  for (Ctx* c : cs) {
    join_user(*c);
    VASMG_CUDA(cudaStreamSynchronize(c->stream));
  }
  // groups: first fit on the per-level region sums
  std::vector<std::vector<int>> groups;
  std::vector<std::vector<int>> load;
  for (int i = 0; i < k; ++i) {
    bool placed = false;
    for (size_t g = 0; g < groups.size() && !placed; ++g) {
      bool fits = true;
      for (int l = 0; l < views[i].lt && fits; ++l)
        fits = (l < (int)load[g].size() ? load[g][l] : 0) + views[i].lv[l].R <= cap;
      if (fits) {
        groups[g].push_back(i);
        if ((int)load[g].size() < views[i].lt) load[g].resize(views[i].lt, 0);
        for (int l = 0; l < views[i].lt; ++l) load[g][l] += views[i].lv[l].R;
        placed = true;
      }
    }
    if (!placed) {
      groups.push_back({i});
      load.push_back(std::vector<int>(views[i].lt));
      for (int l = 0; l < views[i].lt; ++l) load.back()[l] = views[i].lv[l].R;
    }
  }
  int worst = VASMG_OK;
  i64 total = 0;
  cudaStream_t s = cs[0]->stream;
  for (const auto& g : groups) {
    std::vector<EngineView<float>> gv;
    std::vector<const double*> gF;
    std::vector<double*> gU;
    std::vector<vasmg_stats> gst(g.size());
    for (int i : g) {
      gv.push_back(views[i]);
      gF.push_back(F[i]);
      gU.push_back(U[i]);
      if (st) gst[gv.size() - 1] = st[i];
    }
    i64 nl = 0;
    const int rc = sto == 1 ? batch_solve<float>(gv, s, gF.data(), gU.data(), tol, st ? gst.data() : nullptr, &nl)
                            : batch_solve<__nv_bfloat16>(gv, s, gF.data(), gU.data(), tol, st ? gst.data() : nullptr,
                                                         &nl);
    total += nl;
    if (st)
      for (size_t q = 0; q < g.size(); ++q) st[g[q]] = gst[q];
    if (rc < 0) worst = std::min(worst, rc);
    else if (worst >= 0) worst = std::max(worst, rc);
  }
  for (Ctx* c : cs) c->last_launches = total;
  if (launches) *launches = total;
  return worst;
}

double time_kernel_multi(Ctx& c, int which, int level, int k, int reps, double* bytes) {
  return c.eng->time_multi(c, which, level, k, reps, bytes);
}

void lanes_info(Ctx& c, int32_t* g, int n) {
  for (int l = 0; l < n; ++l) g[l] = 0;
  if (c.eng) c.eng->lanes(g, n);
}

void staged_info(Ctx& c, int level, int64_t* v) {
  for (int q = 0; q < 5; ++q) v[q] = 0;
  if (c.eng) c.eng->staged(level, v);
}

// The bounded wait on its own: one CTA waits for a stage word that nothing
// publishes.  The wait must give up after SPIN_LIMIT polls, raise the abort
// flag and return; *result is 1 if the wait was satisfied, 2 if it gave up.
__global__ void wait_probe_kernel(const int* __restrict__ list, const unsigned long long* word, int* abort_flag,
                                  int* result) {
  const bool ok = wait_regions(list, 1, word, 1u, 1u, abort_flag);
  if (threadIdx.x == 0) *result = ok ? 1 : 2;
}

// FP64 FMA throughput: each thread runs FMA_CHAINS independent chains of
// dependent FMAs (enough independent work to cover the FP64 pipe's latency),
// `iters` steps each; the result is stored so the chains are not removed.
constexpr int FMA_CHAINS = 8;
__global__ void __launch_bounds__(256) fp64_fma_kernel(int iters, double* out) {
  double a[FMA_CHAINS];
  const double m = 1.0 - 1e-9 * (double)(threadIdx.x & 7), c = 1e-12 * (double)(blockIdx.x & 15);
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) a[k] = 1.0 + 1e-3 * (double)k + 1e-7 * (double)threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) s += a[k];
  if (s == 12345.678) out[0] = s;  // never true; keeps the chains live
  if (threadIdx.x == 0 && blockIdx.x == 0) out[1] = s;
}

int probe_fp64_rate(double* tflops, double* ms_out) {
  cudaStream_t s = nullptr;
  VASMG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } guard{s};
  int dev = 0, sms = 0, bpsm = 0;
  VASMG_CUDA(cudaGetDevice(&dev));
  VASMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  VASMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, fp64_fma_kernel, 256, 0));
  const int blocks = sms * std::max(1, bpsm), iters = 1 << 14;
  DevBuf<double> out;
  out.alloc(2, s);
  fp64_fma_kernel<<<blocks, 256, 0, s>>>(iters, out.get());  // warm-up
  check_launch("fp64_fma");
  cudaEvent_t e0, e1;
  VASMG_CUDA(cudaEventCreate(&e0));
  VASMG_CUDA(cudaEventCreate(&e1));
  const int reps = 5;
  VASMG_CUDA(cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r) fp64_fma_kernel<<<blocks, 256, 0, s>>>(iters, out.get());
  VASMG_CUDA(cudaEventRecord(e1, s));
  VASMG_CUDA(cudaEventSynchronize(e1));
  float ms = 0.0f;
  VASMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  check_launch("fp64_fma");
  const double per = (double)ms / reps;
  const double flops = 2.0 * FMA_CHAINS * (double)iters * blocks * 256.0;
  if (tflops) *tflops = flops / (per * 1e-3) / 1e12;
  if (ms_out) *ms_out = per;
  return VASMG_OK;
}

int probe_wait_timeout(double* elapsed_ms) {
  cudaStream_t s = nullptr;
  VASMG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } guard{s};
  DevBuf<unsigned long long> word;
  DevBuf<int32_t> list, flags;
  word.alloc(1, s);
  word.zero();
  list.alloc(1, s);
  list.zero();
  flags.alloc(2, s);
  flags.zero();
  cudaEvent_t e0, e1;
  VASMG_CUDA(cudaEventCreate(&e0));
  VASMG_CUDA(cudaEventCreate(&e1));
  VASMG_CUDA(cudaEventRecord(e0, s));
  wait_probe_kernel<<<1, 32, 0, s>>>(list.get(), word.get(), flags.get(), flags.get() + 1);
  check_launch("wait_probe");
  VASMG_CUDA(cudaEventRecord(e1, s));
  VASMG_CUDA(cudaEventSynchronize(e1));
  float ms = 0.0f;
  VASMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (elapsed_ms) *elapsed_ms = ms;
  const std::vector<int32_t> f = flags.download();
  if (f[1] == 2 && f[0] == 1) return VASMG_ERR_TIMEOUT;
  return f[1] == 1 ? VASMG_OK : VASMG_ERR_CUDA;
}

void dense_level_info(Ctx& c, int* kd, int* dn) {
  *kd = -1;
  *dn = 0;
  if (c.eng) c.eng->dense_level(kd, dn);
}

}  // namespace vasmg
