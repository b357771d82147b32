// Device primitives used by the setup: exclusive scan, stable LSD radix sort,
// unique, row pointers from sorted pairs, reductions.  All deterministic.
#include "common.cuh"

namespace vasmg {

// ------------------------------------------------------------------ scan

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T v, T* warp_tot, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  return incl - v + warp_tot[warp];
}

template <typename T>
__global__ void scan_reduce_kernel(const T* __restrict__ in, i64 n, T* __restrict__ sums) {
  __shared__ T wt[32];
  __shared__ T tot;
  i64 base = (i64)blockIdx.x * SCAN_TILE;
  T s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    i64 i = base + (i64)k * SCAN_THREADS + threadIdx.x;
    if (i < n) s += in[i];
  }
  block_exclusive_scan<T>(s, wt, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void scan_apply_kernel(const T* in, T* out, i64 n, const T* __restrict__ offs) {
  __shared__ T tile[SCAN_TILE];
  __shared__ T wt[32];
  __shared__ T tot;
  i64 base = (i64)blockIdx.x * SCAN_TILE;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int j = k * SCAN_THREADS + threadIdx.x;
    i64 i = base + j;
    tile[j] = i < n ? in[i] : T(0);
  }
  __syncthreads();
  T v[SCAN_ITEMS];
  T s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = tile[threadIdx.x * SCAN_ITEMS + k];
    s += v[k];
  }
  T ex = block_exclusive_scan<T>(s, wt, &tot);
  if (offs) ex += offs[blockIdx.x];
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    tile[threadIdx.x * SCAN_ITEMS + k] = ex;
    ex += v[k];
  }
  __syncthreads();
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int j = k * SCAN_THREADS + threadIdx.x;
    i64 i = base + j;
    if (i < n) out[i] = tile[j];
  }
}

template <typename T>
void scan_exclusive(const T* in, T* out, i64 n, cudaStream_t s) {
  if (n <= 0) return;
  i64 nb = ceil_div(n, SCAN_TILE);
  if (nb == 1) {
    scan_apply_kernel<T><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr);
    check_launch("scan_apply");
    return;
  }
  DevBuf<T> sums;
  sums.alloc(nb, s);
  scan_reduce_kernel<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums.get());
  check_launch("scan_reduce");
  scan_exclusive<T>(sums.get(), sums.get(), nb, s);
  scan_apply_kernel<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, sums.get());
  check_launch("scan_apply");
}

void scan_exclusive_i64(const i64* in, i64* out, i64 n, cudaStream_t s) {
  scan_exclusive<long long>((const long long*)in, (long long*)out, n, s);
}
void scan_exclusive_i32(const int32_t* in, int32_t* out, i64 n, cudaStream_t s) { scan_exclusive<int>(in, out, n, s); }

// ------------------------------------------------------------------ radix sort

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_WARPS * RS_ROUNDS * 32;  // 4096 keys per tile

__global__ void rs_hist_kernel(const u64* __restrict__ keys, i64 n, int shift, long long* __restrict__ counts,
                               i64 ntiles) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  i64 base = (i64)blockIdx.x * RS_TILE;
  for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
    i64 i = base + k;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(i64)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: keys of a tile are ranked warp by warp, 32 at a time, with
// __match_any_sync giving each key its rank among equal digits.
template <bool HAS_VAL>
__global__ void __launch_bounds__(RS_THREADS) rs_scatter_kernel(const u64* __restrict__ kin,
                                                                const int32_t* __restrict__ vin,
                                                                u64* __restrict__ kout, int32_t* __restrict__ vout,
                                                                i64 n, int shift,
                                                                const long long* __restrict__ offs, i64 ntiles) {
  __shared__ long long goff[256];
  __shared__ int wcnt[RS_WARPS][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  goff[threadIdx.x] = offs[(i64)threadIdx.x * ntiles + blockIdx.x];
  for (int k = threadIdx.x; k < RS_WARPS * 256; k += RS_THREADS) (&wcnt[0][0])[k] = 0;
  __syncthreads();
  const i64 base = (i64)blockIdx.x * RS_TILE + (i64)warp * (RS_ROUNDS * 32);
  u64 key[RS_ROUNDS];
  int32_t val[RS_ROUNDS];
  int dig[RS_ROUNDS], pos[RS_ROUNDS];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const i64 i = base + r * 32 + lane;
    const bool valid = i < n;
    const u64 k = valid ? kin[i] : 0ull;
    const int d = valid ? (int)((k >> shift) & 255u) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    const int cnt = __popc(peers);
    const int leader = __ffs(peers) - 1;
    const int before = d < 256 ? wcnt[warp][d] : 0;
    __syncwarp();
    if (valid && lane == leader) wcnt[warp][d] = before + cnt;
    __syncwarp();
    key[r] = k;
    if (HAS_VAL) val[r] = valid ? vin[i] : 0;
    dig[r] = d;
    pos[r] = before + rank;
  }
  __syncthreads();
  {
    const int dg = threadIdx.x;
    int run = 0;
    for (int w = 0; w < RS_WARPS; ++w) {
      int t = wcnt[w][dg];
      wcnt[w][dg] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    if (dig[r] < 256) {
      const i64 o = goff[dig[r]] + wcnt[warp][dig[r]] + pos[r];
      kout[o] = key[r];
      if (HAS_VAL) vout[o] = val[r];
    }
  }
}

void radix_sort(u64* keys, int32_t* vals, i64 n, int bits, cudaStream_t s) {
  if (n <= 1) return;
  if (bits <= 0) bits = 1;
  const int passes = (bits + 7) / 8;
  const i64 ntiles = ceil_div(n, RS_TILE);
  DevBuf<u64> kt;
  DevBuf<int32_t> vt;
  DevBuf<long long> counts;
  kt.alloc(n, s);
  if (vals) vt.alloc(n, s);
  counts.alloc(256 * ntiles, s);
  u64* ka = keys;
  u64* kb = kt.get();
  int32_t* va = vals;
  int32_t* vb = vals ? vt.get() : nullptr;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    rs_hist_kernel<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, n, shift, counts.get(), ntiles);
    check_launch("rs_hist");
    scan_exclusive<long long>(counts.get(), counts.get(), 256 * ntiles, s);
    if (vals)
      rs_scatter_kernel<true><<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, counts.get(), ntiles);
    else
      rs_scatter_kernel<false><<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, nullptr, kb, nullptr, n, shift,
                                                                        counts.get(), ntiles);
    check_launch("rs_scatter");
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    VASMG_CUDA(cudaMemcpyAsync(keys, ka, sizeof(u64) * n, cudaMemcpyDeviceToDevice, s));
    if (vals) VASMG_CUDA(cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  }
}

int bits_for(u64 maxval) {
  int b = 0;
  while (b < 64 && (maxval >> b) != 0) ++b;
  return b < 1 ? 1 : b;
}

// ------------------------------------------------------------------ unique / compaction

__global__ void head_flags_kernel(const u64* __restrict__ k, i64 n, long long* __restrict__ f) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    f[i] = (i == 0 || k[i] != k[i - 1]) ? 1 : 0;
}
__global__ void compact_kernel(const u64* __restrict__ k, i64 n, const long long* __restrict__ pos,
                               u64* __restrict__ out) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    if (i == 0 || k[i] != k[i - 1]) out[pos[i]] = k[i];
}

i64 unique_sorted(u64* keys, i64 n, cudaStream_t s) {
  if (n <= 1) return n;
  DevBuf<long long> f;
  f.alloc(n, s);
  head_flags_kernel<<<grid_for(n, 256), 256, 0, s>>>(keys, n, f.get());
  check_launch("head_flags");
  long long last_flag = fetch(f.get() + n - 1, s);
  scan_exclusive<long long>(f.get(), f.get(), n, s);
  long long m = fetch(f.get() + n - 1, s) + last_flag;
  DevBuf<u64> out;
  out.alloc(m, s);
  compact_kernel<<<grid_for(n, 256), 256, 0, s>>>(keys, n, f.get(), out.get());
  check_launch("compact");
  VASMG_CUDA(cudaMemcpyAsync(keys, out.get(), sizeof(u64) * m, cudaMemcpyDeviceToDevice, s));
  VASMG_CUDA(cudaStreamSynchronize(s));
  return m;
}

__global__ void rowptr_kernel(const u64* __restrict__ keys, i64 nnz, i64 nrows, int32_t* __restrict__ rp) {
  for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r <= nrows; r += (i64)gridDim.x * blockDim.x) {
    const u64 target = (u64)r << 32;
    i64 lo = 0, hi = nnz;
    while (lo < hi) {
      i64 mid = (lo + hi) >> 1;
      if (keys[mid] < target) lo = mid + 1; else hi = mid;
    }
    rp[r] = (int32_t)lo;
  }
}

void rowptr_from_pairs(const u64* keys, i64 nnz, i64 nrows, int32_t* rp, cudaStream_t s) {
  rowptr_kernel<<<grid_for(nrows + 1, 256), 256, 0, s>>>(keys, nnz, nrows, rp);
  check_launch("rowptr");
}

// ------------------------------------------------------------------ reductions

__global__ void minmax_kernel(const double* __restrict__ x, i64 n, double* __restrict__ out) {
  __shared__ double smin[256], smax[256];
  double mn = INFINITY, mx = -INFINITY;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    mn = fmin(mn, x[i]);
    mx = fmax(mx, x[i]);
  }
  smin[threadIdx.x] = mn;
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = smin[0];
    out[2 * blockIdx.x + 1] = smax[0];
  }
}

void minmax_f64(const double* x, i64 n, double* mn, double* mx, cudaStream_t s) {
  const int g = grid_for(n, 256, 1024);
  DevBuf<double> part;
  part.alloc(2 * g, s);
  minmax_kernel<<<g, 256, 0, s>>>(x, n, part.get());
  check_launch("minmax");
  std::vector<double> h = part.download();
  double a = INFINITY, b = -INFINITY;
  for (int i = 0; i < g; ++i) {
    a = std::min(a, h[2 * i]);
    b = std::max(b, h[2 * i + 1]);
  }
  *mn = a;
  *mx = b;
}

__global__ void max_i32_kernel(const int32_t* __restrict__ x, i64 n, int* __restrict__ out) {
  int m = INT32_MIN;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) m = max(m, x[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

int32_t max_i32(const int32_t* x, i64 n, cudaStream_t s) {
  DevBuf<int> o;
  o.alloc(1, s);
  int init = INT32_MIN;
  o.upload(&init, 1);
  max_i32_kernel<<<grid_for(n, 256, 2048), 256, 0, s>>>(x, n, o.get());
  check_launch("max_i32");
  return fetch(o.get(), s);
}

__global__ void sum_i64_kernel(const long long* __restrict__ x, i64 n, unsigned long long* __restrict__ out) {
  long long m = 0;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) m += x[i];
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, (unsigned long long)m);
}

i64 sum_i64(const i64* x, i64 n, cudaStream_t s) {
  DevBuf<unsigned long long> o;
  o.alloc(1, s);
  o.zero();
  sum_i64_kernel<<<grid_for(n, 256, 2048), 256, 0, s>>>((const long long*)x, n, o.get());
  check_launch("sum_i64");
  return (i64)fetch(o.get(), s);
}

}  // namespace vasmg
