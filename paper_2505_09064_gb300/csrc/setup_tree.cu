// Region tree, coarse grids and interpolation weights on the device.
//
//  - bounding square (Sec. 3.1.1 Step 1): [m, M]^d with m / M the smallest /
//    largest coordinate over all axes;
//  - the point-region tree of Step 2 (a cell splits while it holds more than T
//    vertices) is not built node by node: the vertices are sorted by Morton key
//    of their quantised coordinates, and each vertex's leaf is the shallowest
//    cell on its path that holds at most T vertices (counted with two binary
//    searches in the sorted keys).  The split rule makes the tree independent
//    of insertion order, so this equals the sequential construction;
//  - Step 3: the non-empty leaves are the level-1 cells, their deduplicated
//    corners the level-1 vertices (sort + unique of lattice keys);
//  - Step 4 / Sec. 3.2: each fine vertex interpolates bilinearly
//    (trilinearly) from the corners of its leaf, w = prod_a (1 - |x_a - c_a|/h);
//  - Sec. 3.1.2: coarser grids by replacing every cell of maximal depth by its
//    parent, until the root; each vertex of a level interpolates from the cell
//    of the next level that contains it (half-open boxes first; on the outer
//    edge of the covered region, the containing closed box of smallest
//    (depth, key)).
//
// All geometric arithmetic is IEEE FP64 with explicit round-to-nearest
// intrinsics (no contraction), in the same order as the CPU oracle, so keys,
// leaves, cells, lattice vertices and weights are bit-identical to it.
#include "common.cuh"

namespace vasmg {

__device__ __forceinline__ double norm_coord(double x, double m, double span) {
  return span > 0.0 ? __ddiv_rn(__dsub_rn(x, m), span) : 0.0;
}

__global__ void morton_keys_kernel(const double* __restrict__ X, i64 nv, int d, int K, double m, double span,
                                   u64* __restrict__ key, u64* __restrict__ skey, int32_t* __restrict__ sval) {
  const double scale = (double)(1ull << K);
  const u64 top = (1ull << K) - 1;
  for (i64 v = (i64)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (i64)gridDim.x * blockDim.x) {
    u64 q[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      const double t = norm_coord(X[v * d + a], m, span);
      const double s = floor(__dmul_rn(t, scale));  // exact: power-of-two scaling
      q[a] = s <= 0.0 ? 0ull : (s >= (double)top ? top : (u64)s);
    }
    const u64 k = morton(q, d);
    key[v] = k;
    skey[v] = k;
    sval[v] = (int32_t)v;
  }
}

__device__ __forceinline__ i64 lower_bound_u64(const u64* __restrict__ a, i64 n, u64 x) {
  i64 lo = 0, hi = n;
  while (lo < hi) {
    i64 mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Count of sorted keys inside the cell of depth `depth` that contains key k.
__device__ __forceinline__ i64 cell_count(const u64* __restrict__ sk, i64 n, u64 k, int depth, int d, int K) {
  const int rest = d * (K - depth);
  const u64 lo = (k >> rest) << rest;
  const u64 hi = lo + (1ull << rest);
  const i64 b = lower_bound_u64(sk, n, lo);
  const i64 e = hi == 0 ? n : lower_bound_u64(sk, n, hi);
  return e - b;
}

__global__ void leaves_kernel(const u64* __restrict__ sk, const int32_t* __restrict__ sv, i64 nv, int d, int K, int T,
                              int32_t* __restrict__ leaf_depth, u64* __restrict__ leaf_start,
                              u64* __restrict__ sorted_leaf_start, int32_t* __restrict__ sorted_leaf_depth) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (i64)gridDim.x * blockDim.x) {
    const u64 k = sk[i];
    // smallest depth whose cell holds <= T vertices (counts shrink with depth)
    int lo = 0, hi = K;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cell_count(sk, nv, k, mid, d, K) <= T) hi = mid; else lo = mid + 1;
    }
    const int rest = d * (K - lo);
    const u64 start = (k >> rest) << rest;
    const int32_t v = sv[i];
    leaf_depth[v] = lo;
    leaf_start[v] = start;
    sorted_leaf_start[i] = start;
    sorted_leaf_depth[i] = lo;
  }
}

// Keep the first of every run of equal starts (starts are sorted).
__global__ void cell_flags_kernel(const u64* __restrict__ st, i64 n, long long* __restrict__ f) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    f[i] = (i == 0 || st[i] != st[i - 1]) ? 1 : 0;
}
__global__ void cell_compact_kernel(const u64* __restrict__ st, const int32_t* __restrict__ dp, i64 n,
                                    const long long* __restrict__ pos, u64* __restrict__ ost,
                                    int32_t* __restrict__ odp) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    if (i == 0 || st[i] != st[i - 1]) {
      ost[pos[i]] = st[i];
      odp[pos[i]] = dp[i];
    }
}

static i64 unique_cells(const u64* st, const int32_t* dp, i64 n, DevBuf<u64>& ost, DevBuf<int32_t>& odp,
                        cudaStream_t s) {
  DevBuf<long long> f;
  f.alloc(n, s);
  cell_flags_kernel<<<grid_for(n, 256), 256, 0, s>>>(st, n, f.get());
  check_launch("cell_flags");
  long long lastf = fetch(f.get() + n - 1, s);
  scan_exclusive_i64((const i64*)f.get(), (i64*)f.get(), n, s);
  i64 m = fetch(f.get() + n - 1, s) + lastf;
  ost.alloc(m, s);
  odp.alloc(m, s);
  cell_compact_kernel<<<grid_for(n, 256), 256, 0, s>>>(st, dp, n, f.get(), ost.get(), odp.get());
  check_launch("cell_compact");
  return m;
}

// Lattice corners (K+1 bits per axis) of every cell, as Morton keys.
__global__ void corner_keys_kernel(const u64* __restrict__ st, const int32_t* __restrict__ dp, i64 ncells, int d,
                                   int K, u64* __restrict__ out) {
  const int nch = 1 << d;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < ncells * nch; i += (i64)gridDim.x * blockDim.x) {
    const i64 cidx = i / nch;
    const int dl = (int)(i - cidx * nch);
    u64 lo[3] = {0, 0, 0};
    unmorton(st[cidx], d, lo);
    const u64 h = 1ull << (K - dp[cidx]);
    u64 p[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) p[a] = lo[a] + (((dl >> a) & 1) ? h : 0ull);
    out[i] = morton(p, d);
  }
}

// Weights of the 2^d corners from local coordinates s_a in [0,1]: the product
// over axes of (1 - s_a) or s_a, multiplied in axis order.
template <int D>
__device__ __forceinline__ void corner_weights(const double* s, double* w) {
#pragma unroll
  for (int dl = 0; dl < (1 << D); ++dl) {
    double acc = 1.0;
#pragma unroll
    for (int a = 0; a < D; ++a) acc = __dmul_rn(acc, ((dl >> a) & 1) ? s[a] : __dsub_rn(1.0, s[a]));
    w[dl] = acc;
  }
}

// One row of an interpolation operator: weights of the corners of the cell
// with low lattice corner `lo` and side h = 2^(K-depth), local coordinates s.
template <int D>
__device__ int interp_row(const u64* lo, u64 h, const double* s, const u64* __restrict__ lat, i64 nlat,
                          int32_t* cols, double* ws) {
  double w[1 << D];
  corner_weights<D>(s, w);
  int m = 0;
#pragma unroll
  for (int dl = 0; dl < (1 << D); ++dl) {
    if (w[dl] == 0.0) continue;
    u64 p[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) p[a] = lo[a] + (((dl >> a) & 1) ? h : 0ull);
    const u64 key = morton(p, D);
    const i64 col = lower_bound_u64(lat, nlat, key);
    // insertion by column index
    int j = m;
    while (j > 0 && cols[j - 1] > (int32_t)col) {
      cols[j] = cols[j - 1];
      ws[j] = ws[j - 1];
      --j;
    }
    cols[j] = (int32_t)col;
    ws[j] = w[dl];
    ++m;
  }
  return m;
}

// P_0: fine vertex -> corners of its leaf; s_a = t_a 2^depth - c_a (exact).
template <int D>
__global__ void p0_kernel(const double* __restrict__ X, i64 nv, int K, double m, double span,
                          const int32_t* __restrict__ leaf_depth, const u64* __restrict__ leaf_start,
                          const u64* __restrict__ lat, i64 nlat, const int32_t* __restrict__ rp,
                          int32_t* __restrict__ cnt, int32_t* __restrict__ ci, double* __restrict__ w) {
  for (i64 v = (i64)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (i64)gridDim.x * blockDim.x) {
    const int dep = leaf_depth[v];
    u64 lo[3] = {0, 0, 0};
    unmorton(leaf_start[v], D, lo);
    const int sh = K - dep;
    double s[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double t = norm_coord(X[v * D + a], m, span);
      s[a] = __dsub_rn(__dmul_rn(t, (double)(1ull << dep)), (double)(lo[a] >> sh));
    }
    int32_t cols[1 << D];
    double ws[1 << D];
    const int k = interp_row<D>(lo, 1ull << sh, s, lat, nlat, cols, ws);
    if (rp == nullptr) {
      cnt[v] = k;
    } else {
      for (int j = 0; j < k; ++j) {
        ci[rp[v] + j] = cols[j];
        w[rp[v] + j] = ws[j];
      }
    }
  }
}

__device__ __forceinline__ i64 upper_bound_u64(const u64* __restrict__ a, i64 n, u64 x) {
  i64 lo = 0, hi = n;
  while (lo < hi) {
    i64 mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Cell (index into the sorted cell list) whose half-open box holds lattice point p, or -1.
template <int D>
__device__ i64 locate_half_open(const u64* p, int K, const u64* __restrict__ st, const int32_t* __restrict__ dp,
                                i64 nc) {
  const u64 lim = 1ull << K;
#pragma unroll
  for (int a = 0; a < D; ++a)
    if (p[a] >= lim) return -1;
  const u64 mk = morton(p, D);
  const i64 idx = upper_bound_u64(st, nc, mk) - 1;
  if (idx < 0) return -1;
  const int rest = D * (K - dp[idx]);
  const u64 size = 1ull << rest;
  return (mk - st[idx]) < size ? idx : -1;
}

template <int D>
__global__ void pl_kernel(const u64* __restrict__ flat, i64 nf, int K, const u64* __restrict__ st,
                          const int32_t* __restrict__ dp, i64 nc, const u64* __restrict__ clat, i64 nclat,
                          const int32_t* __restrict__ rp, int32_t* __restrict__ cnt, int32_t* __restrict__ ci,
                          double* __restrict__ w, int* __restrict__ bad) {
  for (i64 v = (i64)blockIdx.x * blockDim.x + threadIdx.x; v < nf; v += (i64)gridDim.x * blockDim.x) {
    u64 p[3] = {0, 0, 0};
    unmorton(flat[v], D, p);
    i64 cell = locate_half_open<D>(p, K, st, dp, nc);
    if (cell < 0) {
      // outer edge: among the cells whose closed box holds p, the smallest (depth, key)
      int best_depth = 1 << 30;
      u64 best_key = 0;
      for (int dl = 1; dl < (1 << D); ++dl) {
        u64 pp[3] = {0, 0, 0};
        bool ok = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const u64 da = (dl >> a) & 1;
          if (p[a] < da) ok = false;
          pp[a] = p[a] - da;
        }
        if (!ok) continue;
        const i64 c2 = locate_half_open<D>(pp, K, st, dp, nc);
        if (c2 < 0) continue;
        const int dep = dp[c2];
        const u64 key = st[c2] >> (D * (K - dep));
        if (dep < best_depth || (dep == best_depth && key < best_key)) {
          best_depth = dep;
          best_key = key;
          cell = c2;
        }
      }
    }
    if (cell < 0) {
      atomicOr(bad, 1);
      if (rp == nullptr) cnt[v] = 0;
      continue;
    }
    u64 lo[3] = {0, 0, 0};
    unmorton(st[cell], D, lo);
    const int sh = K - dp[cell];
    const double inv = 1.0 / (double)(1ull << sh);  // exact power of two
    double s[D];
#pragma unroll
    for (int a = 0; a < D; ++a) s[a] = __dmul_rn((double)(p[a] - lo[a]), inv);
    int32_t cols[1 << D];
    double ws[1 << D];
    const int k = interp_row<D>(lo, 1ull << sh, s, clat, nclat, cols, ws);
    if (rp == nullptr) {
      cnt[v] = k;
    } else {
      for (int j = 0; j < k; ++j) {
        ci[rp[v] + j] = cols[j];
        w[rp[v] + j] = ws[j];
      }
    }
  }
}

// Sec. 3.1.2: cells at the maximal depth D are replaced by their parents.
__global__ void merge_kernel(const u64* __restrict__ st, const int32_t* __restrict__ dp, i64 n, int D, int d, int K,
                             u64* __restrict__ ost, int32_t* __restrict__ odp) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    if (dp[i] == D) {
      const int rest = d * (K - D + 1);
      ost[i] = rest >= 64 ? 0ull : (st[i] >> rest) << rest;
      odp[i] = D - 1;
    } else {
      ost[i] = st[i];
      odp[i] = dp[i];
    }
  }
}

static void level_vertices(Ctx& c, CanonLevel& lv, const DevBuf<int32_t>& depth) {
  cudaStream_t s = c.stream;
  const int nch = 1 << c.dim;
  const i64 m = lv.ncells * nch;
  DevBuf<u64> keys;
  keys.alloc(m, s);
  corner_keys_kernel<<<grid_for(m, 256), 256, 0, s>>>(lv.cell_start.get(), depth.get(), lv.ncells, c.dim, c.K,
                                                       keys.get());
  check_launch("corner_keys");
  radix_sort(keys.get(), nullptr, m, c.dim * (c.K + 1), s);
  lv.nv = unique_sorted(keys.get(), m, s);
  lv.lat.alloc(lv.nv, s);
  VASMG_CUDA(cudaMemcpyAsync(lv.lat.get(), keys.get(), sizeof(u64) * lv.nv, cudaMemcpyDeviceToDevice, s));
}

static void finish_prolong(Ctx& c, CanonLevel& f, DevBuf<int32_t>& cnt) {
  cudaStream_t s = c.stream;
  f.prp.alloc(f.nv + 1, s);
  scan_exclusive_i32(cnt.get(), f.prp.get(), f.nv + 1, s);
  f.pnnz = fetch(f.prp.get() + f.nv, s);
  f.pci.alloc(f.pnnz, s);
  f.pw.alloc(f.pnnz, s);
}


void setup_tree(Ctx& c) {
  cudaStream_t s = c.stream;
  const int d = c.dim;
  // Step 1: bounding square
  minmax_f64(c.X.get(), c.n, &c.box_m, &c.box_M, s);
  const double span = c.box_M - c.box_m;
  // quantised coordinates -> Morton keys, vertices sorted by key
  c.mkey.alloc(c.nv, s);
  DevBuf<u64> sk;
  sk.alloc(c.nv, s);
  c.morder.alloc(c.nv, s);
  morton_keys_kernel<<<grid_for(c.nv, 256), 256, 0, s>>>(c.X.get(), c.nv, d, c.K, c.box_m, span, c.mkey.get(),
                                                          sk.get(), c.morder.get());
  check_launch("morton_keys");
  radix_sort(sk.get(), c.morder.get(), c.nv, d * c.K, s);
  // Step 2/3: leaves
  DevBuf<int32_t> ldepth;
  ldepth.alloc(c.nv, s);
  c.leaf_start.alloc(c.nv, s);
  DevBuf<u64> sls;
  DevBuf<int32_t> sld;
  sls.alloc(c.nv, s);
  sld.alloc(c.nv, s);
  leaves_kernel<<<grid_for(c.nv, 256), 256, 0, s>>>(sk.get(), c.morder.get(), c.nv, d, c.K, c.T, ldepth.get(),
                                                     c.leaf_start.get(), sls.get(), sld.get());
  check_launch("leaves");
  c.leaf_depth.alloc(c.nv, s);
  {
    std::vector<int32_t> h = ldepth.download();
    std::vector<uint8_t> hb(h.begin(), h.end());
    c.leaf_depth.upload(hb.data(), c.nv);
  }
  c.C.resize(1);
  // a problem small enough for the direct solve has no coarse levels
  if (c.coarse_max_dofs > 0 && c.n <= c.coarse_max_dofs) {
    VASMG_CUDA(cudaStreamSynchronize(s));
    return;
  }
  c.C.emplace_back();
  std::vector<DevBuf<int32_t>> depths(2);
  {
    CanonLevel& L1 = c.C[1];
    L1.ncells = unique_cells(sls.get(), sld.get(), c.nv, L1.cell_start, depths[1], s);
    L1.max_depth = max_i32(depths[1].get(), L1.ncells, s);
    level_vertices(c, L1, depths[1]);
  }
  // P_0
  {
    CanonLevel& L0 = c.C[0];
    CanonLevel& L1 = c.C[1];
    DevBuf<int32_t> cnt;
    cnt.alloc(c.nv + 1, s);
    cnt.zero();
    auto launch = [&](const int32_t* rp) {
      if (d == 2)
        p0_kernel<2><<<grid_for(c.nv, 256), 256, 0, s>>>(c.X.get(), c.nv, c.K, c.box_m, span, ldepth.get(),
                                                          c.leaf_start.get(), L1.lat.get(), L1.nv, rp, cnt.get(),
                                                          L0.pci.get(), L0.pw.get());
      else
        p0_kernel<3><<<grid_for(c.nv, 256), 256, 0, s>>>(c.X.get(), c.nv, c.K, c.box_m, span, ldepth.get(),
                                                          c.leaf_start.get(), L1.lat.get(), L1.nv, rp, cnt.get(),
                                                          L0.pci.get(), L0.pw.get());
      check_launch("p0");
    };
    launch(nullptr);
    finish_prolong(c, L0, cnt);
    launch(L0.prp.get());
  }
  setup_galerkin(c, 0);
  // Sec. 3.1.2: merge the deepest cells until the root
  DevBuf<int> bad;
  bad.alloc(1, s);
  bad.zero();
  while (true) {
    CanonLevel& cur = c.C.back();
    const bool at_root = cur.ncells == 1 && cur.max_depth == 0;
    if (at_root) break;
    if (c.coarse_max_dofs > 0 && cur.nv * d <= c.coarse_max_dofs) break;
    const int l = (int)c.C.size() - 1;
    CanonLevel nx;
    {
      DevBuf<u64> mst;
      DevBuf<int32_t> mdp;
      mst.alloc(cur.ncells, s);
      mdp.alloc(cur.ncells, s);
      merge_kernel<<<grid_for(cur.ncells, 256), 256, 0, s>>>(cur.cell_start.get(), depths[l].get(), cur.ncells,
                                                             cur.max_depth, d, c.K, mst.get(), mdp.get());
      check_launch("merge");
      depths.emplace_back();
      nx.ncells = unique_cells(mst.get(), mdp.get(), cur.ncells, nx.cell_start, depths[l + 1], s);
      nx.max_depth = cur.max_depth - 1;
    }
    level_vertices(c, nx, depths[l + 1]);
    c.C.push_back(std::move(nx));
    CanonLevel& f = c.C[l];
    CanonLevel& g = c.C[l + 1];
    DevBuf<int32_t> cnt;
    cnt.alloc(f.nv + 1, s);
    cnt.zero();
    auto launch = [&](const int32_t* rp) {
      if (d == 2)
        pl_kernel<2><<<grid_for(f.nv, 256), 256, 0, s>>>(f.lat.get(), f.nv, c.K, g.cell_start.get(),
                                                          depths[l + 1].get(), g.ncells, g.lat.get(), g.nv, rp,
                                                          cnt.get(), f.pci.get(), f.pw.get(), bad.get());
      else
        pl_kernel<3><<<grid_for(f.nv, 256), 256, 0, s>>>(f.lat.get(), f.nv, c.K, g.cell_start.get(),
                                                          depths[l + 1].get(), g.ncells, g.lat.get(), g.nv, rp,
                                                          cnt.get(), f.pci.get(), f.pw.get(), bad.get());
      check_launch("pl");
    };
    launch(nullptr);
    finish_prolong(c, f, cnt);
    launch(f.prp.get());
    VASMG_CHECK(fetch(bad.get(), s) == 0, VASMG_ERR_CUDA, "a vertex found no containing cell");
    setup_galerkin(c, l);
  }
  // keep the cell depths as bytes for export
  for (size_t l = 1; l < c.C.size(); ++l) {
    std::vector<int32_t> h = depths[l].download();
    std::vector<uint8_t> hb(h.begin(), h.end());
    c.C[l].cell_depth.alloc(c.C[l].ncells, s);
    c.C[l].cell_depth.upload(hb.data(), c.C[l].ncells);
  }
  VASMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace vasmg
