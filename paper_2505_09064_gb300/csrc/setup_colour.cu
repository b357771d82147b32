// Colouring of every level, colour-contiguous renumbering, and the solve-order
// structures used by the hot path (off-diagonal BSR as value planes, diagonal
// inverses, transfers), plus the dense Cholesky factor of the coarsest level.
//
// Colouring (the smoother of Sec. 2.1 / Alg. 1 run as multicolour point-block
// Gauss-Seidel): Jones-Plassmann rounds; a vertex whose uncoloured neighbours
// all rank lower takes the smallest colour unused by its coloured neighbours.
// Every vertex is coloured after all its higher-ranked neighbours and before
// any lower-ranked one, so the result equals greedy colouring in rank order
// and does not depend on execution order.
// Rank: on the fine level splitmix64(vertex); on coarser levels (lattice
// points) the class sum_a ((p_a / u) mod 3) 3^a first, class 0 highest, with u
// the side of the level's smallest cell, then splitmix64(vertex) >> 6; ties go
// to the smaller vertex.  Uniform coarse levels (radius-2 stencils) then need
// exactly 3^d colours.
#include <algorithm>

#include "common.cuh"

namespace vasmg {

constexpr int MAX_COLOURS = 512;

__device__ __forceinline__ u64 colour_rank(i64 v, const u64* __restrict__ lat, int sh, int d) {
  if (lat == nullptr) return splitmix64((u64)v);
  u64 p[3] = {0, 0, 0};
  unmorton(lat[v], d, p);
  u64 cls = 0, w = 1;
  for (int a = 0; a < d; ++a) {
    cls += ((p[a] >> sh) % 3ull) * w;
    w *= 3;
  }
  return ((w - 1 - cls) << 58) | (splitmix64((u64)v) >> 6);
}

__global__ void jp_round_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, i64 nv,
                                const u64* __restrict__ lat, int sh, int d, const int32_t* __restrict__ cin,
                                int32_t* __restrict__ cout, unsigned long long* __restrict__ remaining,
                                int* __restrict__ overflow) {
  for (i64 v = (i64)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (i64)gridDim.x * blockDim.x) {
    const int32_t cv = cin[v];
    if (cv >= 0) {
      cout[v] = cv;
      continue;
    }
    const u64 pv = colour_rank(v, lat, sh, d);
    u64 used[MAX_COLOURS / 64];
#pragma unroll
    for (int w = 0; w < MAX_COLOURS / 64; ++w) used[w] = 0;
    bool eligible = true;
    for (int32_t k = rp[v]; k < rp[v + 1]; ++k) {
      const int32_t j = ci[k];
      if (j == (int32_t)v) continue;
      const int32_t cj = cin[j];
      if (cj < 0) {
        const u64 pj = colour_rank(j, lat, sh, d);
        if (pj > pv || (pj == pv && j < (int32_t)v)) {
          eligible = false;
          break;
        }
      } else {
        used[cj >> 6] |= 1ull << (cj & 63);
      }
    }
    if (!eligible) {
      cout[v] = -1;
      atomicAdd(remaining, 1ull);
      continue;
    }
    int col = -1;
#pragma unroll
    for (int w = 0; w < MAX_COLOURS / 64; ++w) {
      if (col < 0 && ~used[w] != 0ull) col = w * 64 + __ffsll((long long)~used[w]) - 1;
    }
    if (col < 0) {
      atomicOr(overflow, 1);
      col = 0;
    }
    cout[v] = col;
  }
}

static int colour_level(Ctx& c, CanonLevel& lv, int l) {
  cudaStream_t s = c.stream;
  DevBuf<int32_t> a, b;
  a.alloc(lv.nv, s);
  b.alloc(lv.nv, s);
  VASMG_CUDA(cudaMemsetAsync(a.get(), 0xff, sizeof(int32_t) * lv.nv, s));
  DevBuf<unsigned long long> rem;
  rem.alloc(1, s);
  DevBuf<int> ovf;
  ovf.alloc(1, s);
  ovf.zero();
  for (i64 round = 0; round <= lv.nv; ++round) {
    rem.zero();
    jp_round_kernel<<<grid_for(lv.nv, 256), 256, 0, s>>>(lv.rp.get(), lv.ci.get(), lv.nv,
                                                          l == 0 ? nullptr : lv.lat.get(), c.K - lv.max_depth,
                                                          c.dim, a.get(), b.get(), rem.get(), ovf.get());
    check_launch("jp_round");
    std::swap(a, b);
    if (fetch(rem.get(), s) == 0) break;
  }
  VASMG_CHECK(fetch(ovf.get(), s) == 0, VASMG_ERR_UNSUPPORTED, "more than 512 colours needed");
  lv.colour = std::move(a);
  return max_i32(lv.colour.get(), lv.nv, s) + 1;
}

// ------------------------------------------------------------------ renumbering

__global__ void renum_keys_kernel(const int32_t* __restrict__ colour, const int32_t* __restrict__ secondary, i64 nv,
                                  u64* __restrict__ keys, int32_t* __restrict__ vals) {
  for (i64 v = (i64)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (i64)gridDim.x * blockDim.x) {
    const u64 sec = secondary ? (u64)(uint32_t)secondary[v] : (u64)v;
    keys[v] = ((u64)(uint32_t)colour[v] << 32) | sec;
    vals[v] = (int32_t)v;
  }
}

__global__ void invert_perm_kernel(const int32_t* __restrict__ perm, i64 n, int32_t* __restrict__ iperm) {
  for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (i64)gridDim.x * blockDim.x)
    iperm[perm[r]] = (int32_t)r;
}

__global__ void rank_kernel(const int32_t* __restrict__ order, i64 n, int32_t* __restrict__ rank) {
  for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (i64)gridDim.x * blockDim.x)
    rank[order[r]] = (int32_t)r;
}

// off-diagonal entries keyed by (new row, new col); payload = canonical entry
__global__ void offdiag_keys_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, i64 nv,
                                    const int32_t* __restrict__ iperm, const long long* __restrict__ off,
                                    u64* __restrict__ keys, int32_t* __restrict__ vals) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (i64)gridDim.x * blockDim.x) {
    long long o = off[i];
    const u64 r = (uint32_t)iperm[i];
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int32_t j = ci[k];
      if (j == (int32_t)i) continue;
      keys[o] = (r << 32) | (u64)(uint32_t)iperm[j];
      vals[o] = k;
      ++o;
    }
  }
}

__global__ void row_off_count_kernel(const int32_t* __restrict__ rp, i64 nv, long long* __restrict__ cnt) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (i64)gridDim.x * blockDim.x)
    cnt[i] = rp[i + 1] - rp[i] - 1;
}

__global__ void low32_s_kernel(const u64* __restrict__ k, i64 n, int32_t* __restrict__ out) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    out[i] = (int32_t)(k[i] & 0xffffffffull);
}

__global__ void split_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, i64 nv,
                             int32_t* __restrict__ sp) {
  for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r < nv; r += (i64)gridDim.x * blockDim.x) {
    int32_t lo = rp[r], hi = rp[r + 1];
    while (lo < hi) {
      const int32_t mid = (lo + hi) >> 1;
      if (ci[mid] < (int32_t)r) lo = mid + 1; else hi = mid;
    }
    sp[r] = lo;
  }
}

template <typename S>
__device__ __forceinline__ S cvt_from_double(double v);
template <>
__device__ __forceinline__ double cvt_from_double<double>(double v) { return v; }
template <>
__device__ __forceinline__ float cvt_from_double<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_from_double<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

template <typename S>
__global__ void planes_kernel(const double* __restrict__ cv, const int32_t* __restrict__ ent, i64 nnz, int dd,
                              S* __restrict__ out) {
  for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (i64)gridDim.x * blockDim.x) {
    const double* B = cv + (i64)ent[e] * dd;
    for (int q = 0; q < dd; ++q) out[block_index(q, e, nnz, dd)] = cvt_from_double<S>(B[q]);
  }
}

// Diagonal blocks (level 0, FP64 planes) and their inverses (adjugate / det, FP64).
template <int D>
__global__ void diag_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ cv, const int32_t* __restrict__ perm, i64 nv,
                            double* __restrict__ diag, double* __restrict__ dinv64, float* __restrict__ dinv32,
                            double* __restrict__ cdinv) {
  constexpr int DD = D * D;
  for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r < nv; r += (i64)gridDim.x * blockDim.x) {
    const int32_t i = perm[r];
    int32_t lo = rp[i], hi = rp[i + 1];
    while (lo < hi) {
      const int32_t mid = (lo + hi) >> 1;
      if (ci[mid] < i) lo = mid + 1; else hi = mid;
    }
    const double* B = cv + (i64)lo * DD;
    double inv[DD];
    if (D == 2) {
      const double det = B[0] * B[3] - B[1] * B[2];
      inv[0] = B[3] / det;
      inv[1] = -B[1] / det;
      inv[2] = -B[2] / det;
      inv[3] = B[0] / det;
    } else {
      double cf[9];
      cf[0] = B[4] * B[8] - B[5] * B[7];
      cf[1] = B[5] * B[6] - B[3] * B[8];
      cf[2] = B[3] * B[7] - B[4] * B[6];
      cf[3] = B[2] * B[7] - B[1] * B[8];
      cf[4] = B[0] * B[8] - B[2] * B[6];
      cf[5] = B[1] * B[6] - B[0] * B[7];
      cf[6] = B[1] * B[5] - B[2] * B[4];
      cf[7] = B[2] * B[3] - B[0] * B[5];
      cf[8] = B[0] * B[4] - B[1] * B[3];
      const double det = B[0] * cf[0] + B[1] * cf[1] + B[2] * cf[2];
      // inverse = transpose of the cofactor matrix / det
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) inv[a * 3 + b] = cf[b * 3 + a] / det;
    }
    for (int q = 0; q < DD; ++q) {
      if (diag) diag[(i64)q * nv + r] = B[q];
      if (dinv64) dinv64[(i64)q * nv + r] = inv[q];
      if (dinv32) dinv32[(i64)q * nv + r] = (float)inv[q];
      cdinv[(i64)i * DD + q] = inv[q];
    }
  }
}

// Transfers in solve order: P rows = fine (solve order), columns = coarse (solve order).
template <int D>
__global__ void p_solve_kernel(const int32_t* __restrict__ cprp, const int32_t* __restrict__ cpci,
                               const double* __restrict__ cpw, const int32_t* __restrict__ fperm,
                               const int32_t* __restrict__ ciperm, const int32_t* __restrict__ srp, i64 nf,
                               int32_t* __restrict__ sci, double* __restrict__ w64, float* __restrict__ w32) {
  for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r < nf; r += (i64)gridDim.x * blockDim.x) {
    const int32_t i = fperm[r];
    const int32_t a0 = cprp[i], a1 = cprp[i + 1];
    int32_t cols[1 << D];
    double ws[1 << D];
    int m = 0;
    for (int32_t a = a0; a < a1; ++a) {
      const int32_t col = ciperm[cpci[a]];
      int j = m;
      while (j > 0 && cols[j - 1] > col) {
        cols[j] = cols[j - 1];
        ws[j] = ws[j - 1];
        --j;
      }
      cols[j] = col;
      ws[j] = cpw[a];
      ++m;
    }
    const int32_t o = srp[r];
    for (int j = 0; j < m; ++j) {
      sci[o + j] = cols[j];
      w64[o + j] = ws[j];
      w32[o + j] = (float)ws[j];
    }
  }
}

__global__ void p_rowlen_kernel(const int32_t* __restrict__ cprp, const int32_t* __restrict__ fperm, i64 nf,
                                int32_t* __restrict__ len) {
  for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r < nf; r += (i64)gridDim.x * blockDim.x) {
    const int32_t i = fperm[r];
    len[r] = cprp[i + 1] - cprp[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) len[nf] = 0;
}

__global__ void r_keys_kernel(const int32_t* __restrict__ srp, const int32_t* __restrict__ sci, i64 nf,
                              u64* __restrict__ keys, int32_t* __restrict__ vals) {
  for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r < nf; r += (i64)gridDim.x * blockDim.x)
    for (int32_t a = srp[r]; a < srp[r + 1]; ++a) {
      keys[a] = ((u64)(uint32_t)sci[a] << 32) | (u64)r;
      vals[a] = a;
    }
}

__global__ void r_fill_kernel(const u64* __restrict__ keys, const int32_t* __restrict__ ent, i64 nnz,
                              const double* __restrict__ w64, int32_t* __restrict__ rci, double* __restrict__ rw64,
                              float* __restrict__ rw32) {
  for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += (i64)gridDim.x * blockDim.x) {
    rci[t] = (int32_t)(keys[t] & 0xffffffffull);
    const double w = w64[ent[t]];
    rw64[t] = w;
    rw32[t] = (float)w;
  }
}

__global__ void deadbits_kernel(const uint8_t* __restrict__ dead, const int32_t* __restrict__ perm, i64 nv, int d,
                                uint8_t* __restrict__ bits) {
  for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r < nv; r += (i64)gridDim.x * blockDim.x) {
    const i64 i = perm[r];
    uint8_t b = 0;
    for (int a = 0; a < d; ++a) b |= (dead[i * d + a] ? 1 : 0) << a;
    bits[r] = b;
  }
}

// ------------------------------------------------------------------ coarsest factor

__global__ void dense_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ cv, i64 nv, int d, double* __restrict__ M) {
  const i64 n = nv * d;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (i64)gridDim.x * blockDim.x)
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) M[(i * d + a) * n + (i64)ci[k] * d + b] = cv[(i64)k * d * d + a * d + b];
}

// Left-looking dense Cholesky in canonical order, one CTA.  A pivot at most
// 1e-14 * max diagonal is treated as zero and its direction dropped.
__global__ void cholesky_kernel(double* __restrict__ M, i64 n, uint8_t* __restrict__ drop) {
  __shared__ double maxdiag;
  __shared__ double piv;
  if (threadIdx.x == 0) {
    double md = 0.0;
    for (i64 i = 0; i < n; ++i) md = fmax(md, M[i * n + i]);
    maxdiag = md;
  }
  __syncthreads();
  for (i64 j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double s = M[j * n + j];
      for (i64 k = 0; k < j; ++k) s -= M[j * n + k] * M[j * n + k];
      if (s <= 1e-14 * maxdiag) {
        drop[j] = 1;
        piv = 0.0;
        M[j * n + j] = 0.0;
      } else {
        drop[j] = 0;
        piv = sqrt(s);
        M[j * n + j] = piv;
      }
    }
    __syncthreads();
    for (i64 i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      if (piv == 0.0) {
        M[i * n + j] = 0.0;
        continue;
      }
      double t = M[i * n + j];
      for (i64 k = 0; k < j; ++k) t -= M[i * n + k] * M[j * n + k];
      M[i * n + j] = t / piv;
    }
    __syncthreads();
  }
  // zero the strict upper triangle so only L remains
  for (i64 t = threadIdx.x; t < n * n; t += blockDim.x) {
    const i64 i = t / n, j = t % n;
    if (j > i) M[t] = 0.0;
  }
}

// ------------------------------------------------------------------ driver

void setup_colour_and_solve_levels(Ctx& c) {
  cudaStream_t s = c.stream;
  const int d = c.dim, dd = d * d;
  const int L = (int)c.C.size();
  c.S.clear();
  c.S.resize(L);
  // Morton rank of the fine vertices: the order of vertices inside each colour at level 0
  DevBuf<int32_t> mrank;
  if (c.morder.n == c.nv) {
    mrank.alloc(c.nv, s);
    rank_kernel<<<grid_for(c.nv, 256), 256, 0, s>>>(c.morder.get(), c.nv, mrank.get());
    check_launch("rank");
  }
  for (int l = 0; l < L; ++l) {
    CanonLevel& cl = c.C[l];
    SolveLevel& sl = c.S[l];
    sl.nv = cl.nv;
    cl.ncol = colour_level(c, cl, l);
    sl.ncol = cl.ncol;
    // renumber colour by colour (Morton order inside a colour)
    {
      DevBuf<u64> keys;
      keys.alloc(cl.nv, s);
      sl.perm.alloc(cl.nv, s);
      renum_keys_kernel<<<grid_for(cl.nv, 256), 256, 0, s>>>(cl.colour.get(), l == 0 && mrank.n ? mrank.get() : nullptr,
                                                              cl.nv, keys.get(), sl.perm.get());
      check_launch("renum_keys");
      radix_sort(keys.get(), sl.perm.get(), cl.nv, 32 + bits_for((u64)cl.ncol), s);
      sl.iperm.alloc(cl.nv, s);
      invert_perm_kernel<<<grid_for(cl.nv, 256), 256, 0, s>>>(sl.perm.get(), cl.nv, sl.iperm.get());
      check_launch("invert_perm");
      std::vector<u64> hk = keys.download();
      sl.sec.resize(hk.size());
      for (size_t i = 0; i < hk.size(); ++i) sl.sec[i] = (uint32_t)hk[i];
      sl.cs.assign(cl.ncol + 1, 0);
      for (int col = 0; col <= cl.ncol; ++col) {
        const u64 t = (u64)col << 32;
        sl.cs[col] = (int32_t)(std::lower_bound(hk.begin(), hk.end(), t) - hk.begin());
      }
    }
    // off-diagonal blocks in solve order, columns ascending
    {
      DevBuf<long long> cnt;
      cnt.alloc(cl.nv + 1, s);
      cnt.zero();
      row_off_count_kernel<<<grid_for(cl.nv, 256), 256, 0, s>>>(cl.rp.get(), cl.nv, cnt.get());
      check_launch("row_off_count");
      scan_exclusive_i64((const i64*)cnt.get(), (i64*)cnt.get(), cl.nv + 1, s);
      sl.nnz = fetch(cnt.get() + cl.nv, s);
      DevBuf<u64> keys;
      DevBuf<int32_t> ent;
      keys.alloc(sl.nnz, s);
      ent.alloc(sl.nnz, s);
      offdiag_keys_kernel<<<grid_for(cl.nv, 256), 256, 0, s>>>(cl.rp.get(), cl.ci.get(), cl.nv, sl.iperm.get(),
                                                                cnt.get(), keys.get(), ent.get());
      check_launch("offdiag_keys");
      radix_sort(keys.get(), ent.get(), sl.nnz, 32 + bits_for((u64)cl.nv), s);
      sl.rp.alloc(cl.nv + 1, s);
      sl.ci.alloc(sl.nnz, s);
      sl.sp.alloc(cl.nv, s);
      rowptr_from_pairs(keys.get(), sl.nnz, cl.nv, sl.rp.get(), s);
      low32_s_kernel<<<grid_for(sl.nnz, 256), 256, 0, s>>>(keys.get(), sl.nnz, sl.ci.get());
      check_launch("low32");
      split_kernel<<<grid_for(cl.nv, 256), 256, 0, s>>>(sl.rp.get(), sl.ci.get(), cl.nv, sl.sp.get());
      check_launch("split");
      sl.ent = std::move(ent);
    }
    sl.deadbits.alloc(cl.nv, s);
    deadbits_kernel<<<grid_for(cl.nv, 256), 256, 0, s>>>(cl.dead.get(), sl.perm.get(), cl.nv, d, sl.deadbits.get());
    check_launch("deadbits");
  }
  // transfers in solve order
  for (int l = 0; l + 1 < L; ++l) {
    CanonLevel& cf = c.C[l];
    SolveLevel& sf = c.S[l];
    SolveLevel& sg = c.S[l + 1];
    DevBuf<int32_t> len;
    len.alloc(sf.nv + 1, s);
    p_rowlen_kernel<<<grid_for(sf.nv, 256), 256, 0, s>>>(cf.prp.get(), sf.perm.get(), sf.nv, len.get());
    check_launch("p_rowlen");
    sf.prp.alloc(sf.nv + 1, s);
    scan_exclusive_i32(len.get(), sf.prp.get(), sf.nv + 1, s);
    sf.pci.alloc(cf.pnnz, s);
    sf.pw64.alloc(cf.pnnz, s);
    sf.pw32.alloc(cf.pnnz, s);
    if (d == 2)
      p_solve_kernel<2><<<grid_for(sf.nv, 256), 256, 0, s>>>(cf.prp.get(), cf.pci.get(), cf.pw.get(), sf.perm.get(),
                                                              sg.iperm.get(), sf.prp.get(), sf.nv, sf.pci.get(),
                                                              sf.pw64.get(), sf.pw32.get());
    else
      p_solve_kernel<3><<<grid_for(sf.nv, 256), 256, 0, s>>>(cf.prp.get(), cf.pci.get(), cf.pw.get(), sf.perm.get(),
                                                              sg.iperm.get(), sf.prp.get(), sf.nv, sf.pci.get(),
                                                              sf.pw64.get(), sf.pw32.get());
    check_launch("p_solve");
    DevBuf<u64> keys;
    DevBuf<int32_t> ent;
    keys.alloc(cf.pnnz, s);
    ent.alloc(cf.pnnz, s);
    r_keys_kernel<<<grid_for(sf.nv, 256), 256, 0, s>>>(sf.prp.get(), sf.pci.get(), sf.nv, keys.get(), ent.get());
    check_launch("r_keys");
    radix_sort(keys.get(), ent.get(), cf.pnnz, 32 + bits_for((u64)sg.nv), s);
    sf.rrp.alloc(sg.nv + 1, s);
    rowptr_from_pairs(keys.get(), cf.pnnz, sg.nv, sf.rrp.get(), s);
    sf.rci.alloc(cf.pnnz, s);
    sf.rw64.alloc(cf.pnnz, s);
    sf.rw32.alloc(cf.pnnz, s);
    r_fill_kernel<<<grid_for(cf.pnnz, 256), 256, 0, s>>>(keys.get(), ent.get(), cf.pnnz, sf.pw64.get(), sf.rci.get(),
                                                          sf.rw64.get(), sf.rw32.get());
    check_launch("r_fill");
  }
  solve_level_values(c);
  VASMG_CUDA(cudaStreamSynchronize(s));
}

// Values of every level in solve order -- off-diagonal planes in the
// precisions the solve needs, diagonal blocks and their inverses -- and the
// coarsest Cholesky factor.  Buffers are allocated on the first call and
// refilled in place afterwards (the solve engine keeps their addresses).
void solve_level_values(Ctx& c) {
  cudaStream_t s = c.stream;
  const int d = c.dim, dd = d * d;
  const int L = (int)c.C.size();
  auto ensure = [&](auto& buf, i64 n) {
    if (buf.n != n) buf.alloc(n, s);
  };
  for (int l = 0; l < L; ++l) {
    CanonLevel& cl = c.C[l];
    SolveLevel& sl = c.S[l];
    const bool need64 = l == 0 || c.precision == VASMG_FP64;
    if (need64) {
      ensure(sl.off64, (i64)dd * sl.nnz);
      planes_kernel<double><<<grid_for(sl.nnz, 256), 256, 0, s>>>(cl.v.get(), sl.ent.get(), sl.nnz, dd,
                                                                   sl.off64.get());
      check_launch("planes64");
    }
    if (c.precision == VASMG_FP32_VCYCLE) {
      ensure(sl.off32, (i64)dd * sl.nnz);
      planes_kernel<float><<<grid_for(sl.nnz, 256), 256, 0, s>>>(cl.v.get(), sl.ent.get(), sl.nnz, dd,
                                                                  sl.off32.get());
      check_launch("planes32");
    }
    if (c.precision == VASMG_FP32_VCYCLE_BF16_SMOOTH) {
      ensure(sl.off16, (i64)dd * sl.nnz);
      planes_kernel<__nv_bfloat16><<<grid_for(sl.nnz, 256), 256, 0, s>>>(cl.v.get(), sl.ent.get(), sl.nnz, dd,
                                                                           sl.off16.get());
      check_launch("planes16");
    }
    // level 0 (the SELL operator) and, for the W-cycle's coarse residuals, every level
    const bool keep_diag = l == 0 || c.gamma >= 2;
    if (keep_diag) ensure(sl.diag64, (i64)dd * cl.nv);
    ensure(sl.dinv64, (i64)dd * cl.nv);
    ensure(sl.dinv32, (i64)dd * cl.nv);
    ensure(cl.dinv, (i64)dd * cl.nv);
    if (d == 2)
      diag_kernel<2><<<grid_for(cl.nv, 256), 256, 0, s>>>(cl.rp.get(), cl.ci.get(), cl.v.get(), sl.perm.get(), cl.nv,
                                                           keep_diag ? sl.diag64.get() : nullptr, sl.dinv64.get(),
                                                           sl.dinv32.get(), cl.dinv.get());
    else
      diag_kernel<3><<<grid_for(cl.nv, 256), 256, 0, s>>>(cl.rp.get(), cl.ci.get(), cl.v.get(), sl.perm.get(), cl.nv,
                                                           keep_diag ? sl.diag64.get() : nullptr, sl.dinv64.get(),
                                                           sl.dinv32.get(), cl.dinv.get());
    check_launch("diag");
  }
  // coarsest dense Cholesky (canonical order of the last level)
  CanonLevel& cl = c.C[L - 1];
  c.nc = cl.nv * d;
  VASMG_CHECK(c.nc <= 4096, VASMG_ERR_UNSUPPORTED, "coarsest level larger than 4096 dofs");
  ensure(c.chol, c.nc * c.nc);
  c.chol.zero();
  ensure(c.chol_drop, c.nc);
  dense_kernel<<<grid_for(cl.nv, 64), 64, 0, s>>>(cl.rp.get(), cl.ci.get(), cl.v.get(), cl.nv, d, c.chol.get());
  check_launch("dense");
  cholesky_kernel<<<1, 1024, 0, s>>>(c.chol.get(), c.nc, c.chol_drop.get());
  check_launch("cholesky");
}

}  // namespace vasmg
