// Device building blocks of the solve path shared by the translation units
// that launch it (solve.cu: the single right-hand-side engine; solve_multi.cu:
// several right-hand sides per launch): constants, the level views, the row
// passes of the multicolour sweeps and residuals, the bounded region waits,
// the transfers, the coarsest solve, the cluster tail and the FP64 CG kernels.
#pragma once

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace vasmg {

constexpr int TAIL_NV = 20000;
constexpr int TAIL_THREADS = 1024;
constexpr int TAIL_G = 8;
// lanes per row in the tail: 3D coarse rows hold ~100 blocks
template <int D>
constexpr int tail_g() { return D == 2 ? TAIL_G : 32; }
constexpr int ONE_CTA_NV = 1200;  // tail levels this small run on one CTA
// Dynamic shared memory the tail kernel is configured for.  The limit is an
// attribute of the kernel function, shared by every handle in the process, so
// every engine sets the same value once instead of its own size: a handle
// with a smaller tail would otherwise lower the limit under another one.
constexpr int TAIL_SMEM_MAX = 200 * 1024;
constexpr int MAX_LEVELS = 40;
// The dense level (FP32 vectors only): the first level of the one-CTA tail
// part whose order n satisfies n^2 <= (CTAs of the tail cluster) *
// DENSE_ROWS_PER_CTA^2; the cluster reads M once per V-cycle.
constexpr int DENSE_ROWS_PER_CTA = 640;
constexpr int CG_THREADS = 256;
// Threads of a region CTA of the single-vector sweeps: 1024 (one CTA per SM,
// 152 larger regions) for 2D levels with FP32 vectors, 256 otherwise.
// Measured per solve: 2D 1024^2 FP32 57.0 -> 52.8 ms with 1024; the 3D
// levels (~100 blocks per row) need more than 64 registers per thread and
// are slower with it (128^3 graded: 555 -> 862 ms).
template <int D, typename V>
constexpr int df_threads() { return (D == 2 && sizeof(V) == 4) ? 1024 : 256; }
constexpr int REGION_MIN_ROWS = 32;  // fewest rows a sweep region is given
constexpr int SPIN_LIMIT = 1 << 20;   // ~0.1-0.5 s of polling before a wait gives up

struct Scalars {
  double rho, pq, alpha, beta, rr, res0, relres, tol;
  int iter, max_iters, done, status, first, bodies, abort, pad;
  unsigned int cnt[4];
};

// per-level launch state: exit counters and epochs of the down and up launches
enum { C_DEXIT = 0, C_DEPOCH, C_UEXIT, C_UEPOCH, C_N };

// ------------------------------------------------------------------ memory helpers

template <typename V, typename S>
__device__ __forceinline__ V ldv(const S* p);
template <>
__device__ __forceinline__ double ldv<double, double>(const double* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ldv<float, float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ldv<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
// A 2 x 2 block stored contiguously (4 values): one 16-byte load for FP32,
// two for FP64, one 8-byte load for BF16.
template <typename V, typename S>
__device__ __forceinline__ void ldv4(const S* p, V (&a)[4]) {
  if constexpr (std::is_same<S, float>::value) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    a[0] = t.x, a[1] = t.y, a[2] = t.z, a[3] = t.w;
  } else if constexpr (std::is_same<S, double>::value) {
    const double2 t0 = __ldg(reinterpret_cast<const double2*>(p));
    const double2 t1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
    a[0] = t0.x, a[1] = t0.y, a[2] = t1.x, a[3] = t1.y;
  } else {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&t.x);
    const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&t.y);
    a[0] = __low2float(lo), a[1] = __high2float(lo), a[2] = __low2float(hi), a[3] = __high2float(hi);
  }
}

// Components 0..7 of a 3 x 3 block, stored contiguously: one 16-byte load
// for BF16, two for FP32, four for FP64.
template <typename V, typename S, int N>
__device__ __forceinline__ void ldv8(const S* p, V (&a)[N]) {
  static_assert(N >= 8, "a 3 x 3 block");
  if constexpr (std::is_same<S, float>::value) {
    const float4 t0 = __ldg(reinterpret_cast<const float4*>(p));
    const float4 t1 = __ldg(reinterpret_cast<const float4*>(p) + 1);
    a[0] = t0.x, a[1] = t0.y, a[2] = t0.z, a[3] = t0.w, a[4] = t1.x, a[5] = t1.y, a[6] = t1.z, a[7] = t1.w;
  } else if constexpr (std::is_same<S, double>::value) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const double2 t = __ldg(reinterpret_cast<const double2*>(p) + h);
      a[2 * h] = t.x, a[2 * h + 1] = t.y;
    }
  } else {
    const uint4 t = __ldg(reinterpret_cast<const uint4*>(p));
    const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const __nv_bfloat162 v2 = *reinterpret_cast<const __nv_bfloat162*>(&w[h]);
      a[2 * h] = __low2float(v2), a[2 * h + 1] = __high2float(v2);
    }
  }
}

// vectors written inside a launch by other CTAs are read from L2 (.cg)
// LC: the vector is produced and consumed by one CTA only, so plain (L1-cached)
// accesses are coherent after a CTA barrier.
template <bool LC = false, typename V>
__device__ __forceinline__ V ldx(const V* p) {
  if constexpr (LC) return *p;
  else return __ldcg(p);
}
template <bool LC = false, typename V>
__device__ __forceinline__ void stx(V* p, V v) {
  if constexpr (LC) *p = v;
  else __stcg(p, v);
}
// A vector value written inside the launch by other CTAs: from L2 (.cg), or
// (L1) through the SM's L1 cache.  L1 is used only by the region launches,
// whose every colour step starts after a GPU-scope acquire (the neighbour
// wait), which invalidates the SM's L1: a cached value is then never older
// than the last step's, and within a step no value a row reads is written
// (rows of one colour are not neighbours).  Rows of a region share most of
// their neighbours, so their gathers mostly hit L1.
template <bool L1, typename T>
__device__ __forceinline__ T ld_shared_vec(const T* p) {
  if constexpr (L1) return __ldca(p);
  else return __ldcg(p);
}

// The D components of one vertex from global memory: one 8- or 16-byte load
// for D = 2 (rows of 2 values are aligned to their size), a pair and a
// single for D = 3 unless PAIR3 is false (the region sweeps: measured slower
// there); one load per component from shared memory.
template <int D, bool LC = false, bool PAIR3 = true, bool L1 = false, typename V>
__device__ __forceinline__ void ldx_vertex(const V* p, V (&v)[D]) {
  if constexpr (D == 2 && !LC && std::is_same<V, float>::value) {
    const float2 t = ld_shared_vec<L1>(reinterpret_cast<const float2*>(p));
    v[0] = t.x;
    v[1] = t.y;
  } else if constexpr (D == 2 && !LC && std::is_same<V, double>::value) {
    const double2 t = ld_shared_vec<L1>(reinterpret_cast<const double2*>(p));
    v[0] = t.x;
    v[1] = t.y;
  } else if constexpr (D == 3 && !LC && PAIR3 && (std::is_same<V, float>::value || std::is_same<V, double>::value)) {
    // 3 values: a pair on its 2-value boundary and a single (the vectors
    // start on a 256-byte boundary, so the parity of the element index says
    // which pair is aligned)
    using V2 = typename std::conditional<std::is_same<V, float>::value, float2, double2>::type;
    if (((reinterpret_cast<uintptr_t>(p) / sizeof(V)) & 1) == 0) {
      const V2 t = ld_shared_vec<L1>(reinterpret_cast<const V2*>(p));
      v[0] = t.x;
      v[1] = t.y;
      v[2] = ld_shared_vec<L1>(p + 2);
    } else {
      v[0] = ld_shared_vec<L1>(p);
      const V2 t = ld_shared_vec<L1>(reinterpret_cast<const V2*>(p + 1));
      v[1] = t.x;
      v[2] = t.y;
    }
  } else if constexpr (!LC) {
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = ld_shared_vec<L1>(p + a);
  } else {
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = ldx<LC>(p + a);
  }
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ------------------------------------------------------------------ level view

template <typename V>
struct LV {
  int nv, ncol;
  long long nnz;
  const int* rp;
  const int* ci;
  const int* sp;          // first entry of a later colour in each row
  const void* off;        // off-diagonal blocks of S, layout block_index()
  // the same blocks split by part, each part contiguous: lower = columns of
  // earlier colours, upper = later colours (the sweeps and the residual read
  // only the part they need)
  const int* rpl;
  const int* cil;
  const void* offl;       // lower part, layout block_index() with n = nlo
  long long nlo;
  const int* rph;
  const int* cih;
  const void* offh;       // upper part, layout block_index() with n = nhi
  long long nhi;
  const V* dinv;          // planes [d*d][nv]
  const uint8_t* dead;    // per vertex, bit a = component a removed
  V* x;
  V* b;
  V* r;
  const int* cs;          // colour starts [ncol+1]
  // transfer to level l+1
  int nvc;
  const int* prp;
  const int* pci;
  const V* pw;
  const int* rrp;
  const int* rci;
  const V* rw;
  V* bc;                  // b of level l+1
  const V* xc;            // x of level l+1
  // region decomposition: CTA k of a sweep launch owns region k, the rows
  // whose spatial key lies in the k-th of R equal key ranges
  int R;
  const int* RS;          // [ncol][R+1]: rows of colour c in region k = [RS[c][k], RS[c][k+1])
  const int* nb_rp;       // regions holding a neighbour of a row of region k (CSR, k excluded)
  const int* nb;
  unsigned long long* pg_d;  // progress of each region in the down launch: epoch << 32 | stage
  unsigned long long* pg_u;  // same for the up launch
  int* ctr;               // C_N counters
};

template <int D>
__device__ __forceinline__ double pick(const double (&a)[D], int i) {
  return D == 2 ? (i == 0 ? a[0] : a[1]) : (i == 0 ? a[0] : (i == 1 ? a[1] : a[D - 1]));
}
template <int D>
__device__ __forceinline__ float pick(const float (&a)[D], int i) {
  return D == 2 ? (i == 0 ? a[0] : a[1]) : (i == 0 ? a[0] : (i == 1 ? a[1] : a[D - 1]));
}

// Entries of one row as a contiguous segment A[a0 .. a0 + len) of the arrays
// the level and mode select (b0 / B are kept for a second segment and unused).
struct RowSeg {
  int a0, la, b0, len;
};

// A level with split parts (LV): MODE 0 reads the lower part, MODE 2 the
// upper part, MODE 1 (whole rows) the combined arrays; one segment each.
template <int MODE, typename S, typename V>
__device__ __forceinline__ void seg_ptrs(const LV<V>& L, const int*& ciA, const S*& offA, long long& nA,
                                         const int*& ciB, const S*& offB, long long& nB) {
  if (MODE == 2) {
    ciA = L.cih;
    offA = (const S*)L.offh;
    nA = L.nhi;
  } else if (MODE == 0) {
    ciA = L.cil;
    offA = (const S*)L.offl;
    nA = L.nlo;
  } else {
    ciA = L.ci;
    offA = (const S*)L.off;
    nA = L.nnz;
  }
  ciB = ciA;
  offB = offA;
  nB = nA;
}
template <int MODE, typename V>
__device__ __forceinline__ RowSeg seg_range(const LV<V>& L, int row) {
  const int* p = MODE == 2 ? L.rph : (MODE == 0 ? L.rpl : L.rp);
  RowSeg r;
  r.a0 = __ldg(p + row);
  r.la = __ldg(p + row + 1) - r.a0;
  r.b0 = 0;
  r.len = r.la;
  return r;
}

// Column index and d x d block of entry e of a row.
template <int D, typename V, typename S>
__device__ __forceinline__ int seg_entry(const RowSeg& r, int e, const int* ciA, const S* offA, long long nA,
                                         const int* ciB, const S* offB, long long nB, V (&a)[D * D]) {
  // every caller passes a single segment (la == len): B is never read
  const int k = r.a0 + e;
  const int* cp = ciA;
  const S* op = offA;
  const long long n = nA;
  (void)ciB;
  (void)offB;
  (void)nB;
  if constexpr (D == 2) {
    (void)n;
    ldv4<V, S>(op + (long long)k * 4, a);  // 2D blocks are stored contiguously
  } else {
    ldv8<V, S>(op + (long long)k * 8, a);  // components 0..7 contiguous (block_index)
    a[8] = ldv<V, S>(op + 8 * n + k);
  }
  return __ldg(cp + k);
}

// Gathers of a region level go through L1 (see ld_shared_vec); the cluster
// tail's levels keep L2 loads.
template <typename V>
struct TL;
template <typename L_t>
struct is_tail_level : std::false_type {};
template <typename V>
struct is_tail_level<TL<V>> : std::true_type {};
template <typename L_t, bool LC>
constexpr bool gather_l1() { return !LC && !is_tail_level<L_t>::value; }

// acc += sum over the row entries e = e0, e0 + G, ... < len of A_e x_{col(e)},
// one entry at a time.  PAIR3: 3D vertex values gathered as an aligned pair
// and a single (see ldx_vertex).  (Loading several entries before their
// gathers was measured: no faster for the sweeps, which wait at their
// barriers, and twice as slow for the residual, whose occupancy it halved.)
template <int D, int G, typename V, typename S, int MODE, bool LC, bool PAIR3, typename L_t>
__device__ __forceinline__ void row_entries(const L_t& L, const RowSeg& sg, int e0, V (&acc)[D]) {
  const int* ciA;
  const S* offA;
  long long nA;
  const int* ciB;
  const S* offB;
  long long nB;
  seg_ptrs<MODE, S>(L, ciA, offA, nA, ciB, offB, nB);
  for (int e = e0; e < sg.len; e += G) {
    V blk[D * D];
    const int j = seg_entry<D, V, S>(sg, e, ciA, offA, nA, ciB, offB, nB, blk);
    V xj[D];
    ldx_vertex<D, LC, PAIR3, gather_l1<L_t, LC>()>((const V*)L.x + (long long)j * D, xj);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int bb = 0; bb < D; ++bb) acc[a] += blk[a * D + bb] * xj[bb];
  }
}

// One row of a sweep / residual by a group of G lanes.
// MODE 0: x_i = Dinv (b_i - lower part), MODE 1: x_i = Dinv (b_i - all
// off-diagonal blocks), MODE 2: r_i = -(upper part).
template <int D, int G, typename V, typename S, int MODE, typename L_t, bool LC = false>
__device__ __forceinline__ void row_pass(const L_t& L, int row, bool valid, int lane) {
  RowSeg sg{0, 0, 0, 0};
  if (valid) sg = seg_range<MODE>(L, row);
  V acc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) acc[a] = V(0);
  row_entries<D, G, V, S, MODE, LC, true>(L, sg, lane, acc);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o, G);
  if (!valid || lane >= D) return;
  if (MODE == 2) {
    stx<LC>(L.r + (long long)row * D + lane, -pick<D>(acc, lane));
  } else {
    V s = V(0);
#pragma unroll
    for (int bb = 0; bb < D; ++bb)
      s += __ldg((const V*)L.dinv + (long long)(lane * D + bb) * L.nv + row) *
           (ldx<LC>((const V*)L.b + (long long)row * D + bb) - acc[bb]);
    stx<LC>(L.x + (long long)row * D + lane, s);
  }
}

// Entries a lane keeps in registers between the prefetch and the finish of a row.
template <int D, typename V, int NPF_ = ((D * D * sizeof(V) <= 16) ? 2 : 1)>
struct RowPF {
  static constexpr int NPF = NPF_;
  RowSeg sg;
  int cj[NPF];
  V a[NPF][D * D];
  V di[D], bv[D];
};

// Row pass split in two.  row_prefetch loads everything that nothing writes
// during the sweep (row range, the first NPF entries of this lane, the
// diagonal inverse and b); row_finish, called once the rows this row depends
// on are done, gathers x and completes the row as row_pass does.
template <int D, int G, typename V, typename S, int MODE, typename L_t, bool LC = false, int NPF>
__device__ __forceinline__ void row_prefetch(const L_t& L, int row, bool valid, int lane, RowPF<D, V, NPF>& st) {
  st.sg = RowSeg{0, 0, 0, 0};
  if (valid) st.sg = seg_range<MODE>(L, row);
  const int* ciA;
  const S* offA;
  long long nA;
  const int* ciB;
  const S* offB;
  long long nB;
  seg_ptrs<MODE, S>(L, ciA, offA, nA, ciB, offB, nB);
#pragma unroll
  for (int p = 0; p < NPF; ++p) {
    const int e = lane + p * G;
    st.cj[p] = -1;
    if (e < st.sg.len) st.cj[p] = seg_entry<D, V, S>(st.sg, e, ciA, offA, nA, ciB, offB, nB, st.a[p]);
  }
  if (MODE != 2 && valid && lane < D) {
#pragma unroll
    for (int bb = 0; bb < D; ++bb) {
      st.di[bb] = __ldg((const V*)L.dinv + (long long)(lane * D + bb) * L.nv + row);
      st.bv[bb] = ldx<LC>((const V*)L.b + (long long)row * D + bb);
    }
  }
}

template <int D, int G, typename V, typename S, int MODE, typename L_t, bool LC = false, int NPF>
__device__ __forceinline__ void row_finish(const L_t& L, int row, bool valid, int lane, const RowPF<D, V, NPF>& st) {
  V acc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) acc[a] = V(0);
#pragma unroll
  for (int p = 0; p < NPF; ++p) {
    if (st.cj[p] >= 0) {
      V xj[D];
      ldx_vertex<D, LC, false, gather_l1<L_t, LC>()>((const V*)L.x + (long long)st.cj[p] * D, xj);
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int bb = 0; bb < D; ++bb) acc[a] += st.a[p][a * D + bb] * xj[bb];
    }
  }
  row_entries<D, G, V, S, MODE, LC, false>(L, st.sg, lane + NPF * G, acc);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o, G);
  if (!valid || lane >= D) return;
  if (MODE == 2) {
    stx<LC>(L.r + (long long)row * D + lane, -pick<D>(acc, lane));
  } else {
    V s = V(0);
#pragma unroll
    for (int bb = 0; bb < D; ++bb) s += st.di[bb] * (st.bv[bb] - acc[bb]);
    stx<LC>(L.x + (long long)row * D + lane, s);
  }
}

template <int D, typename V, typename L_t, bool LC = false>
__device__ __forceinline__ void restrict_row(const L_t& L, int I) {
  V acc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) acc[a] = V(0);
  // four entries' indices, weights and gathers in flight at a time; the sums
  // in entry order (the multi and batched restrictions add in the same order)
  const int t0 = __ldg(L.rrp + I), t1 = __ldg(L.rrp + I + 1);
  int t = t0;
  for (; t + 4 <= t1; t += 4) {
    int ii[4];
    V ww[4], rr[4][D];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ii[u] = __ldg(L.rci + t + u);
      ww[u] = __ldg((const V*)L.rw + t + u);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      ldx_vertex<D, LC, true, gather_l1<L_t, LC>()>((const V*)L.r + (long long)ii[u] * D, rr[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] += ww[u] * rr[u][a];
  }
  for (; t < t1; ++t) {
    const int i = __ldg(L.rci + t);
    const V w = __ldg((const V*)L.rw + t);
    V ri[D];
    ldx_vertex<D, LC, true, gather_l1<L_t, LC>()>((const V*)L.r + (long long)i * D, ri);
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] += w * ri[a];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) stx<LC>((V*)L.bc + (long long)I * D + a, acc[a]);
}

template <int D, typename V, typename L_t, bool LC = false>
__device__ __forceinline__ void prolong_row(const L_t& L, int i) {
  V acc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) acc[a] = V(0);
  // four entries in flight at a time, the sums in entry order (as restrict_row)
  const int t0 = __ldg(L.prp + i), t1 = __ldg(L.prp + i + 1);
  int t = t0;
  for (; t + 4 <= t1; t += 4) {
    int jj[4];
    V ww[4], xx[4][D];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      jj[u] = __ldg(L.pci + t + u);
      ww[u] = __ldg((const V*)L.pw + t + u);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      ldx_vertex<D, LC, true, gather_l1<L_t, LC>()>((const V*)L.xc + (long long)jj[u] * D, xx[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] += ww[u] * xx[u][a];
  }
  for (; t < t1; ++t) {
    const int J = __ldg(L.pci + t);
    const V w = __ldg((const V*)L.pw + t);
    V xJ[D];
    ldx_vertex<D, LC, true, gather_l1<L_t, LC>()>((const V*)L.xc + (long long)J * D, xJ);
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] += w * xJ[a];
  }
  const uint8_t dm = __ldg(L.dead + i);
#pragma unroll
  for (int a = 0; a < D; ++a)
    if (!((dm >> a) & 1)) {
      V* px = (V*)L.x + (long long)i * D + a;
      stx<LC>(px, ldx<LC>((const V*)px) + acc[a]);
    }
}

// ------------------------------------------------------------------ region progress

// Barrier of the NT threads 0..NT-1 of the CTA (named barrier 1), or of the
// whole CTA when NT is 0.
template <int NT = 0>
__device__ __forceinline__ void part_sync() {
  if constexpr (NT == 0) __syncthreads();
  else asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// Wait until every region in list[0..n) has published stage >= need in this
// launch (epoch); false (uniform over the threads 0..NT-1, or the CTA) if a
// wait gave up or the abort flag is up.  Warp 0 polls, one neighbour per
// lane, with GPU-scope acquire loads and back-off.  The acquire that sees a
// neighbour's stage synchronises with that neighbour's release, and the
// barrier after the polls orders it before every thread's reads.  (A full
// fence.acq_rel.gpu after relaxed polls also waits for warp 0's own earlier
// stores to land: the region kernels took 4.7 % longer with it.)
template <int NT = 0>
__device__ __forceinline__ bool wait_regions(const int* __restrict__ list, int n, const unsigned long long* pg,
                                             unsigned epoch, unsigned need, int* abort_flag) {
  __shared__ int s_ok;
  if (threadIdx.x < 32) {
    bool ok = true;
    for (int k = threadIdx.x; k < n && ok; k += 32) {
      const unsigned long long* f = pg + __ldg(list + k);
      int spins = 0;
      unsigned ns = 32;
      for (;;) {
        const unsigned long long v = ld_acquire64(f);
        if ((unsigned)(v >> 32) == epoch && (unsigned)v >= need) break;
        if (++spins > SPIN_LIMIT || *(volatile int*)abort_flag) {
          atomicExch(abort_flag, 1);
          ok = false;
          break;
        }
        __nanosleep(ns);
        ns = ns < 256 ? 2 * ns : 256;
      }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (threadIdx.x == 0) s_ok = ok ? 1 : 0;
  }
  part_sync<NT>();
  return s_ok != 0;
}

// Publish this region's stage once every thread of the CTA (or every one of
// its threads 0..NT-1, the ones that write) has written: the barrier orders
// their writes before thread 0's release, and a release is cumulative, so a
// CTA that acquires the stage sees all of them.
template <int NT = 0>
__device__ __forceinline__ void publish_stage(unsigned long long* f, unsigned epoch, unsigned stage) {
  part_sync<NT>();
  if (threadIdx.x == 0) st_release64(f, ((unsigned long long)epoch << 32) | stage);
}

// The last CTA to leave advances the launch's epoch (nctas: the CTAs sharing
// these counters; the grid unless several levels share one launch).
__device__ __forceinline__ void leave(int* ctr, int exit_i, int epoch_i, int nctas = -1) {
  __syncthreads();
  if (nctas < 0) nctas = (int)gridDim.x;
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ctr + exit_i, 1) == nctas - 1) {
      ctr[exit_i] = 0;
      ctr[epoch_i] += 1;
      __threadfence();
    }
  }
}

// Rows [r0, r1) of one colour, NG rows per pass; the next pass's entries are
// loaded while the current pass gathers x.  `cur` holds the first pass.
template <int D, int G, typename V, typename S, int MODE>
__device__ __forceinline__ void rows_pipelined(const LV<V>& L, int r0, int r1, RowPF<D, V>& cur) {
  constexpr int NG = df_threads<D, V>() / G;
  const int g = threadIdx.x / G, lane = threadIdx.x & (G - 1);
  for (int base = r0; base < r1; base += NG) {
    const int nb = base + NG;
    RowPF<D, V> nxt;
    if (nb < r1) row_prefetch<D, G, V, S, MODE>(L, nb + g, nb + g < r1, lane, nxt);
    row_finish<D, G, V, S, MODE>(L, base + g, base + g < r1, lane, cur);
    if (nb < r1) cur = nxt;
  }
}

// ------------------------------------------------------------------ down / up launches
//
// One cooperative launch per level and direction, CTA k = region k.  A
// region runs its rows colour by colour; before colour c it waits until every
// neighbouring region has finished the colours it reads (forward: all
// earlier colours; backward: all later colours and the prolongation).  The
// neighbour relation is symmetric, so the same waits also keep a region from
// overwriting values a neighbour has still to read.

// Minimum resident CTAs per SM the kernels are compiled for (register cap).
template <int D, typename V>
constexpr int df_min_blocks() { return (D == 2 && sizeof(V) == 4) ? 1 : 2; }

// Forward multicolour sweep from zero (pre-smoothing) of one level.
template <int D, int G, typename V, typename S>
__global__ void __launch_bounds__(df_threads<D, V>(), df_min_blocks<D, V>())
    vdown_kernel(const __grid_constant__ LV<V> L, Scalars* sc) {
  __shared__ unsigned s_epoch;
  if (threadIdx.x == 0) s_epoch = *(volatile unsigned*)(L.ctr + C_DEPOCH);
  __syncthreads();
  const unsigned epoch = s_epoch;
  const int k = blockIdx.x, R = L.R, C = L.ncol;
  const int g = threadIdx.x / G, lane = threadIdx.x & (G - 1);
  const int nb0 = __ldg(L.nb_rp + k), nnb = __ldg(L.nb_rp + k + 1) - nb0;
  int* abort_flag = &sc->abort;
  unsigned long long* mine = L.pg_d + k;
  for (int c = 0; c < C; ++c) {
    const int r0 = __ldg(L.RS + c * (R + 1) + k), r1 = __ldg(L.RS + c * (R + 1) + k + 1);
    if (r0 < r1) {
      RowPF<D, V> cur;
      row_prefetch<D, G, V, S, 0>(L, r0 + g, r0 + g < r1, lane, cur);
      if (c > 0 && !wait_regions(L.nb + nb0, nnb, L.pg_d, epoch, (unsigned)c, abort_flag)) break;
      rows_pipelined<D, G, V, S, 0>(L, r0, r1, cur);
    }
    publish_stage(mine, epoch, (unsigned)(c + 1));
  }
  leave(L.ctr, C_DEXIT, C_DEPOCH);
}

// Backward multicolour sweep (post-smoothing) of one level.
template <int D, int G, typename V, typename S>
__global__ void __launch_bounds__(df_threads<D, V>(), df_min_blocks<D, V>())
    vup_kernel(const __grid_constant__ LV<V> L, Scalars* sc) {
  __shared__ unsigned s_epoch;
  if (threadIdx.x == 0) s_epoch = *(volatile unsigned*)(L.ctr + C_UEPOCH);
  __syncthreads();
  const unsigned epoch = s_epoch;
  const int k = blockIdx.x, R = L.R, C = L.ncol;
  const int g = threadIdx.x / G, lane = threadIdx.x & (G - 1);
  const int nb0 = __ldg(L.nb_rp + k), nnb = __ldg(L.nb_rp + k + 1) - nb0;
  int* abort_flag = &sc->abort;
  unsigned long long* mine = L.pg_u + k;
  unsigned stage = 0;
  for (int c = C - 1; c >= 0; --c) {
    const int r0 = __ldg(L.RS + c * (R + 1) + k), r1 = __ldg(L.RS + c * (R + 1) + k + 1);
    if (r0 < r1) {
      RowPF<D, V> cur;
      row_prefetch<D, G, V, S, 1>(L, r0 + g, r0 + g < r1, lane, cur);
      if (stage > 0 && !wait_regions(L.nb + nb0, nnb, L.pg_u, epoch, stage, abort_flag)) break;
      rows_pipelined<D, G, V, S, 1>(L, r0, r1, cur);
    }
    publish_stage(mine, epoch, ++stage);
  }
  leave(L.ctr, C_UEXIT, C_UEPOCH);
}

// r = -(upper part) x after the zero-start forward sweep: a plain SpMV of
// the later-colour blocks, G lanes per row, grid-strided over the rows.
// The residual of one row of a region level (row_pass, MODE 2) with each lane's
// entries taken two at a time: both blocks and both gathers in flight before
// the products, which are added in entry order.  The kernel keeps 32 registers
// with FP32 vectors (8 CTAs per SM): 128^3 graded, level-1 residual
// 312 -> 291 us.
template <int D, int G, typename V, typename S>
__device__ __forceinline__ void residual_row_u2(const LV<V>& L, int row, bool valid, int lane) {
  RowSeg sg{0, 0, 0, 0};
  if (valid) sg = seg_range<2>(L, row);
  V acc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) acc[a] = V(0);
  const int* ciA;
  const S* offA;
  long long nA;
  const int* ciB;
  const S* offB;
  long long nB;
  seg_ptrs<2, S>(L, ciA, offA, nA, ciB, offB, nB);
  int e = lane;
  for (; e + G < sg.len; e += 2 * G) {
    V b0[D * D], b1[D * D];
    const int j0 = seg_entry<D, V, S>(sg, e, ciA, offA, nA, ciB, offB, nB, b0);
    const int j1 = seg_entry<D, V, S>(sg, e + G, ciA, offA, nA, ciB, offB, nB, b1);
    V x0[D], x1[D];
    ldx_vertex<D, false, true, true>((const V*)L.x + (long long)j0 * D, x0);
    ldx_vertex<D, false, true, true>((const V*)L.x + (long long)j1 * D, x1);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int bb = 0; bb < D; ++bb) acc[a] += b0[a * D + bb] * x0[bb];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int bb = 0; bb < D; ++bb) acc[a] += b1[a * D + bb] * x1[bb];
  }
  if (e < sg.len) {
    V b0[D * D];
    const int j0 = seg_entry<D, V, S>(sg, e, ciA, offA, nA, ciB, offB, nB, b0);
    V x0[D];
    ldx_vertex<D, false, true, true>((const V*)L.x + (long long)j0 * D, x0);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int bb = 0; bb < D; ++bb) acc[a] += b0[a * D + bb] * x0[bb];
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o, G);
  if (!valid || lane >= D) return;
  stx<false>(L.r + (long long)row * D + lane, -pick<D>(acc, lane));
}
template <int D, int G, typename V, typename S>
__global__ void __launch_bounds__(256, sizeof(V) == 8 ? 6 : 8) residual_kernel(const __grid_constant__ LV<V> L) {
  constexpr int NG = 256 / G;
  const int g = threadIdx.x / G, lane = threadIdx.x & (G - 1);
  for (int base = blockIdx.x * NG; base < L.nv; base += gridDim.x * NG)
    residual_row_u2<D, G, V, S>(L, base + g, base + g < L.nv, lane);
}

// b_{l+1} = R r_l (one thread per coarse row)
template <int D, typename V>
__global__ void __launch_bounds__(256) restrict_kernel(const __grid_constant__ LV<V> L) {
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < L.nvc; I += gridDim.x * blockDim.x) restrict_row<D, V>(L, I);
}

// x_l += P x_{l+1} (one thread per fine row)
template <int D, typename V>
__global__ void __launch_bounds__(256) prolong_kernel(const __grid_constant__ LV<V> L) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.nv; i += gridDim.x * blockDim.x) prolong_row<D, V>(L, i);
}

// ------------------------------------------------------------------ staged region sweeps (3D)
//
// The region sweeps of 3D levels with the operator part they read streamed
// through shared memory.  Within one colour step of a region, each group of G
// lanes takes a list of the step's rows, one row after another; lane e of a
// group takes the row's entries e, e + G, e + 2G, ... (as row_finish does)
// and the group sums its lanes by the same shuffle tree.  So each thread runs
// through a stream of slots, ceil(len / G) (at least one) per row of its
// group.  Each such level keeps the part a sweep reads (forward: the lower
// part, backward: whole rows) a second time, in stream order: chunk t of a
// step holds, for each of the step's first nact consumer threads (the warps
// its rows keep busy), its slots EPT t .. EPT t + EPT - 1 (EPT = stg_ept:
// the column, flagged on the last slot of a row, and the block).
// The rows are dealt to the groups longest first, each to the group with the
// fewest slots so far, so the streams of a step end close together and the
// chunks are nearly full.  A producer warp copies a region's chunks ahead,
// with bulk asynchronous copies, into a ring of shared-memory stages (an
// mbarrier per stage counts the bytes in, another counts the consumer warps
// out).  It needs no neighbour data, so it fills the ring while the rows
// wait for their neighbours, and the rows' critical path keeps only the
// gathers of x.  Every row's arithmetic, and its order, is that of
// row_finish: the results are bitwise those of the unstaged sweep (and so of
// the multi and batched sweeps).

constexpr int STG_T = 256;  // consumer threads of a staged sweep CTA; one producer warp follows them
// a slot: column in bits 0..29 (STG_NONE: no entry), STG_END: the row ends
// with this slot; -1: padding after the thread's stream
constexpr int STG_NONE = 0x3fffffff;
constexpr int STG_END = 0x40000000;

// slots per consumer thread and chunk (as many gathers in flight): 4 with
// BF16 or FP32 blocks, 2 with FP64 (128^3 graded, region sweeps: 3.8 % and
// 4.5 % faster than 2 and 1)
template <typename S>
constexpr int stg_ept() { return sizeof(S) == 8 ? 2 : 4; }
// bytes of one chunk of nact threads: the slots, then block components 0..7,
// then component 8 (a multiple of 16 for any nact that is a multiple of 32)
template <typename S>
constexpr int stg_chunk_bytes(int nact = STG_T) { return nact * stg_ept<S>() * (4 + 9 * (int)sizeof(S)); }
// ring stages: at most 96 KB of shared memory per CTA (two CTAs per SM), at
// least two
template <typename S>
constexpr int stg_stages() { return std::min(8, std::max(2, (96 * 1024) / stg_chunk_bytes<S>())); }
template <typename S>
constexpr int stg_smem_bytes() { return stg_stages<S>() * stg_chunk_bytes<S>(); }

template <typename S>
struct StagedOp {
  const int* ci;                // per step, per chunk: [EPT][nact] slots
  const S* v8;                  // [EPT][nact][8] block components 0..7 (same slot order)
  const S* v9;                  // [EPT][nact] block component 8
  const long long* step_off;    // [ncol R + 1]: first slot of colour c in region k (step c R + k)
  const int* step_nact;         // [ncol R]: consumer threads the step's chunks hold (a multiple of 32)
  const int* goff;              // [ncol R][NG + 1]: rows of group g in a step: srow[r0 + goff[g] .. r0 + goff[g + 1])
  const int* srow;              // [nv]: each step's rows [r0, r1), group by group
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait for the phase of the given parity to complete.  Gives up (false)
// after SPIN_LIMIT polls (after the first 64, 64 ns apart), raising the abort
// flag, or soon after another wait raised it (read every 256 polls; never
// when abort_flag is null).
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, int* abort_flag) {
  for (int spins = 0;; ++spins) {
    if (mbar_test(b, parity)) return true;
    if (spins >= SPIN_LIMIT) {
      if (abort_flag) atomicExch(abort_flag, 1);
      return false;
    }
    if (spins >= 64) __nanosleep(64);
    if (abort_flag && (spins & 255) == 255 && *(volatile int*)abort_flag) return false;
  }
}
// bytes from global src to this CTA's shared dst, counted on mbarrier b
// (both addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(b))
               : "memory");
}

// The same with an L2 cache policy (createpolicy), e.g. evict-first for a
// stream read once so that the vectors gathered beside it stay in L2.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, unsigned bytes, unsigned long long* b,
                                              unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Block components of slot `slot` of a chunk of ne slots in shared memory,
// converted as ldv8 / ldv do.
template <typename V, typename S>
__device__ __forceinline__ void stg_block(const unsigned char* chunk, int ne, int slot, V (&a)[9]) {
  const S* p8 = reinterpret_cast<const S*>(chunk + ne * 4) + slot * 8;
  const S* p9 = reinterpret_cast<const S*>(chunk + ne * (4 + 8 * (int)sizeof(S))) + slot;
  if constexpr (std::is_same<S, float>::value) {
    const float4 t0 = reinterpret_cast<const float4*>(p8)[0];
    const float4 t1 = reinterpret_cast<const float4*>(p8)[1];
    a[0] = t0.x, a[1] = t0.y, a[2] = t0.z, a[3] = t0.w, a[4] = t1.x, a[5] = t1.y, a[6] = t1.z, a[7] = t1.w;
    a[8] = *p9;
  } else if constexpr (std::is_same<S, double>::value) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const double2 t = reinterpret_cast<const double2*>(p8)[h];
      a[2 * h] = t.x, a[2 * h + 1] = t.y;
    }
    a[8] = *p9;
  } else {
    const uint4 t = *reinterpret_cast<const uint4*>(p8);
    const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const __nv_bfloat162 v2 = *reinterpret_cast<const __nv_bfloat162*>(&w[h]);
      a[2 * h] = __low2float(v2), a[2 * h + 1] = __high2float(v2);
    }
    a[8] = __bfloat162float(*p9);
  }
}

// The producer: region k's chunks in sweep order into the ring.  EVICT_FIRST:
// the copies mark the operator stream evict-first in L2 (the multi-RHS
// sweeps, whose gathered vectors are KR times larger).
template <typename S, int MODE, bool EVICT_FIRST = false>
__device__ __forceinline__ void stg_produce(const StagedOp<S>& O, int k, int R, int C, unsigned long long* full,
                                            unsigned long long* empty, unsigned char* ring, int* abort_flag) {
  constexpr int NS = stg_stages<S>(), CB = stg_chunk_bytes<S>(), EPT = stg_ept<S>();
  unsigned long long pol = 0;
  if constexpr (EVICT_FIRST) pol = l2_evict_first_policy();
  long long q = 0;  // chunks issued
  bool ok = true;
  for (int i = 0; i < C && ok; ++i) {
    const int c = MODE == 0 ? i : C - 1 - i, step = c * R + k;
    const long long e0 = __ldg(O.step_off + step), e1 = __ldg(O.step_off + step + 1);
    const int ne = EPT * __ldg(O.step_nact + step);  // slots of one chunk of this step
    for (long long e = e0; e < e1; e += ne, ++q) {
      const int s = (int)(q % NS);
      if (q >= NS && !mbar_wait(&empty[s], (unsigned)((q / NS - 1) & 1), abort_flag)) {
        ok = false;
        break;
      }
      unsigned char* dst = ring + s * CB;
      mbar_arrive_tx(&full[s], (unsigned)(ne * (4 + 9 * (int)sizeof(S))));
      if constexpr (EVICT_FIRST) {
        bulk_g2s_hint(dst, O.ci + e, ne * 4, &full[s], pol);
        bulk_g2s_hint(dst + ne * 4, O.v8 + e * 8, ne * 8 * (int)sizeof(S), &full[s], pol);
        bulk_g2s_hint(dst + ne * (4 + 8 * (int)sizeof(S)), O.v9 + e, ne * (int)sizeof(S), &full[s], pol);
      } else {
        bulk_g2s(dst, O.ci + e, ne * 4, &full[s]);
        bulk_g2s(dst + ne * 4, O.v8 + e * 8, ne * 8 * (int)sizeof(S), &full[s]);
        bulk_g2s(dst + ne * (4 + 8 * (int)sizeof(S)), O.v9 + e, ne * (int)sizeof(S), &full[s]);
      }
    }
  }
  // the copies still in flight land before the CTA leaves (after an abort
  // the consumers stop taking chunks)
  for (long long j = q > NS ? q - NS : 0; j < q; ++j) mbar_wait(&full[j % NS], (unsigned)((j / NS) & 1), nullptr);
}

// Diagonal inverse row and b of a row (lanes a < D of its group).
template <int D, typename V>
__device__ __forceinline__ void stg_row_data(const LV<V>& L, int row, bool load, int lane, V (&di)[D], V (&bv)[D]) {
  if (load) {
#pragma unroll
    for (int bb = 0; bb < D; ++bb) {
      di[bb] = __ldg((const V*)L.dinv + (long long)(lane * D + bb) * L.nv + row);
      bv[bb] = ldx<false>((const V*)L.b + (long long)row * D + bb);
    }
  }
}

// The consumers: region k's rows colour by colour, each group of G lanes
// through its rows' slots, chunk by chunk from the ring.
template <int D, int G, typename V, typename S, int MODE>
__device__ __forceinline__ void stg_consume(const LV<V>& L, const StagedOp<S>& O, int k, int R, int C,
                                            unsigned epoch, unsigned long long* full, unsigned long long* empty,
                                            const unsigned char* ring, int* abort_flag) {
  constexpr int NS = stg_stages<S>(), CB = stg_chunk_bytes<S>(), EPT = stg_ept<S>();
  constexpr int NG = STG_T / G;
  const int tid = threadIdx.x, g = tid / G, lane = tid & (G - 1);
  // the lanes of this group within the warp
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((tid & 31) & ~(G - 1)));
  const int nb0 = __ldg(L.nb_rp + k), nnb = __ldg(L.nb_rp + k + 1) - nb0;
  unsigned long long* pg = MODE == 0 ? L.pg_d : L.pg_u;
  long long q = 0;  // chunks taken
  for (int i = 0; i < C; ++i) {
    const int c = MODE == 0 ? i : C - 1 - i;
    const int r0 = __ldg(L.RS + c * (R + 1) + k), r1 = __ldg(L.RS + c * (R + 1) + k + 1);
    if (r0 < r1) {
      const int step = c * R + k;
      // this group's rows: srow[j0 .. j1)
      int j = r0 + __ldg(O.goff + (long long)step * (NG + 1) + g);
      const int j1 = r0 + __ldg(O.goff + (long long)step * (NG + 1) + g + 1);
      // the current row, the next (its diagonal inverse and b in flight) and
      // the one after (its index in flight)
      int row = j < j1 ? __ldg(O.srow + j) : -1;
      int rown = j + 1 < j1 ? __ldg(O.srow + j + 1) : -1;
      int rown2 = j + 2 < j1 ? __ldg(O.srow + j + 2) : -1;
      V di[D], bv[D], dn[D], bn[D];
      stg_row_data<D, V>(L, row, row >= 0 && lane < D, lane, di, bv);
      stg_row_data<D, V>(L, rown, rown >= 0 && lane < D, lane, dn, bn);
      if (i > 0 && !wait_regions<STG_T>(L.nb + nb0, nnb, pg, epoch, (unsigned)i, abort_flag)) break;
      const int nact = __ldg(O.step_nact + step), ne = EPT * nact;
      const long long nch = (__ldg(O.step_off + step + 1) - __ldg(O.step_off + step)) / ne;
      V acc[D];
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] = V(0);
      for (long long t = 0; t < nch; ++t, ++q) {
        const int s = (int)(q % NS);
        // a wait that gave up leaves the chunk unread by the whole warp, so a
        // lane group never splits between taking and skipping it
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[s], (unsigned)((q / NS) & 1), abort_flag));
        const unsigned char* chunk = ring + s * CB;
        int v[EPT];
        V xj[EPT][D];
#pragma unroll
        for (int h = 0; h < EPT; ++h) {
          v[h] = ok && tid < nact ? reinterpret_cast<const int*>(chunk)[h * nact + tid] : -1;
          const int col = v[h] & STG_NONE;
          if (v[h] >= 0 && col != STG_NONE)
            ldx_vertex<D, false, false, true>((const V*)L.x + (long long)col * D, xj[h]);
        }
#pragma unroll
        for (int h = 0; h < EPT; ++h) {
          if (v[h] < 0) continue;
          if ((v[h] & STG_NONE) != STG_NONE) {
            V blk[9];
            stg_block<V, S>(chunk, ne, h * nact + tid, blk);
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
              for (int bb = 0; bb < D; ++bb) acc[a] += blk[a * D + bb] * xj[h][bb];
          }
          if (v[h] & STG_END) {
            // the row is done: the group's sum, x_row, the next row
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
              for (int a = 0; a < D; ++a) acc[a] += __shfl_xor_sync(gmask, acc[a], o, G);
            if (row >= 0 && lane < D) {
              V sum = V(0);
#pragma unroll
              for (int bb = 0; bb < D; ++bb) sum += di[bb] * (bv[bb] - acc[bb]);
              stx<false>(L.x + (long long)row * D + lane, sum);
            }
#pragma unroll
            for (int a = 0; a < D; ++a) acc[a] = V(0);
            ++j;
            row = rown;
            rown = rown2;
#pragma unroll
            for (int bb = 0; bb < D; ++bb) di[bb] = dn[bb], bv[bb] = bn[bb];
            stg_row_data<D, V>(L, rown, rown >= 0 && lane < D, lane, dn, bn);
            rown2 = j + 2 < j1 ? __ldg(O.srow + j + 2) : -1;
          }
        }
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[s]);
      }
    }
    publish_stage<STG_T>(pg + k, epoch, (unsigned)(i + 1));
  }
}

// Forward sweep from zero (MODE 0, lower part) or backward sweep (MODE 1,
// whole rows) of a 3D region level with the staged operator: the waits and
// stages of vdown_kernel / vup_kernel.
template <int D, int G, typename V, typename S, int MODE>
__global__ void __launch_bounds__(STG_T + 32, 2)
    vstaged_kernel(const __grid_constant__ LV<V> L, const __grid_constant__ StagedOp<S> O, Scalars* sc) {
  static_assert(D == 3, "the staged layout holds 3 x 3 blocks");
  constexpr int NS = stg_stages<S>();
  extern __shared__ __align__(128) unsigned char stg_ring[];
  __shared__ __align__(8) unsigned long long full[NS], empty[NS];
  __shared__ unsigned s_epoch;
  if (threadIdx.x == 0) {
    s_epoch = *(volatile unsigned*)(L.ctr + (MODE == 0 ? C_DEPOCH : C_UEPOCH));
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], STG_T / 32);
    }
    mbar_fence_init();
  }
  __syncthreads();
  const unsigned epoch = s_epoch;
  const int k = blockIdx.x;
  int* abort_flag = &sc->abort;
  if (threadIdx.x >= STG_T) {
    if (threadIdx.x == STG_T) stg_produce<S, MODE>(O, k, L.R, L.ncol, full, empty, stg_ring, abort_flag);
  } else {
    stg_consume<D, G, V, S, MODE>(L, O, k, L.R, L.ncol, epoch, full, empty, stg_ring, abort_flag);
  }
  leave(L.ctr, MODE == 0 ? C_DEXIT : C_UEXIT, MODE == 0 ? C_DEPOCH : C_UEPOCH);
}

// Fills the staged copy of one part (rows rp / columns ci / blocks off with n
// blocks, layout block_index): one thread per step and consumer thread
// writes that thread's stream and the padding after it.
template <typename S>
__global__ void stage_fill_kernel(const int* __restrict__ rp, const int* __restrict__ ci, const S* __restrict__ off,
                                  long long n, const int* __restrict__ RS, int R, int C,
                                  const long long* __restrict__ step_off, const int* __restrict__ step_nact,
                                  const int* __restrict__ goff, const int* __restrict__ srow, int G,
                                  int* __restrict__ sci, S* __restrict__ sv8, S* __restrict__ sv9) {
  constexpr int EPT = stg_ept<S>();
  const int NG = STG_T / G;
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < (long long)C * R * STG_T;
       w += (long long)gridDim.x * blockDim.x) {
    const int step = (int)(w / STG_T), tid = (int)(w - (long long)step * STG_T);
    const int nact = step_nact[step];
    if (tid >= nact) continue;  // no rows: the step's chunks leave this thread out
    const int c = step / R, k = step - c * R;
    const int g = tid / G, lane = tid % G;
    const int r0 = RS[c * (R + 1) + k];
    const long long e0 = step_off[step], nslots = (step_off[step + 1] - e0) / nact;
    long long pos = 0;
    auto put = [&](int v, long long kk) {
      const long long slot = e0 + (pos / EPT) * EPT * nact + (pos % EPT) * nact + tid;
      sci[slot] = v;
#pragma unroll
      for (int q = 0; q < 8; ++q) sv8[slot * 8 + q] = kk >= 0 ? off[kk * 8 + q] : S(0.0f);
      sv9[slot] = kk >= 0 ? off[8 * n + kk] : S(0.0f);
      ++pos;
    };
    for (int j = r0 + goff[(long long)step * (NG + 1) + g]; j < r0 + goff[(long long)step * (NG + 1) + g + 1]; ++j) {
      const int row = srow[j];
      const int a0 = rp[row], len = rp[row + 1] - a0;
      const int steps = len > 0 ? (len + G - 1) / G : 1;
      for (int t = 0; t < steps; ++t) {
        const int e = t * G + lane;
        const int end = t == steps - 1 ? STG_END : 0;
        if (e < len) put(ci[a0 + e] | end, a0 + e);
        else put(STG_NONE | end, -1);
      }
    }
    while (pos < nslots) put(-1, -1);
  }
}

// ------------------------------------------------------------------ coarsest solve and tail

struct CoarseArgs {
  const double* chol;      // n x n lower factor, canonical dof order
  const uint8_t* drop;
  const int* perm;         // solve index -> canonical vertex (coarsest level)
  double* y;               // scratch [n]
  int n, d;
};

// Forward / backward substitution with the Cholesky factor, by one warp:
// gather b into canonical order, substitute, scatter back to solve order.
template <typename V, bool LC = false>
__device__ void coarse_solve_warp(const CoarseArgs& A, const V* b, V* x) {
  const int lane = threadIdx.x & 31;
  const int n = A.n, d = A.d;
  for (int t = lane; t < n; t += 32) {
    const int r = t / d, a = t - r * d;
    A.y[(long long)__ldg(A.perm + r) * d + a] = (double)ldx<LC>(b + t);
  }
  __syncwarp();
  chol_substitute_warp(A.chol, A.drop, n, A.y);
  for (int t = lane; t < n; t += 32) {
    const int r = t / d, a = t - r * d;
    stx<LC>(x + t, (V)A.y[(long long)__ldg(A.perm + r) * d + a]);
  }
}

template <typename V>
__global__ void coarse_kernel(CoarseArgs A, const V* b, V* x) {
  if (threadIdx.x < 32) coarse_solve_warp<V>(A, b, x);
}

// A level as the tail kernel sees it (the fields row_pass and the transfers use).
template <typename V>
struct TL {
  int nv;
  long long nnz;
  const int* rp;
  const int* ci;
  const int* sp;
  const void* off;
  const V* dinv;
  const uint8_t* dead;
  V* x;
  V* b;
  V* r;
  const int* cs;
  int ncol, nvc;
  const int* prp;
  const int* pci;
  const V* pw;
  const int* rrp;
  const int* rci;
  const V* rw;
  V* bc;
  const V* xc;
};

// A tail level keeps the combined CSR: one segment, [rp, sp) lower, [sp,
// rp+1) upper.
template <int MODE, typename S, typename V>
__device__ __forceinline__ void seg_ptrs(const TL<V>& L, const int*& ciA, const S*& offA, long long& nA,
                                         const int*& ciB, const S*& offB, long long& nB) {
  ciA = ciB = L.ci;
  offA = offB = (const S*)L.off;
  nA = nB = L.nnz;
}
template <int MODE, typename V>
__device__ __forceinline__ RowSeg seg_range(const TL<V>& L, int row) {
  RowSeg r;
  r.a0 = MODE == 2 ? __ldg(L.sp + row) : __ldg(L.rp + row);
  const int a1 = MODE == 0 ? __ldg(L.sp + row) : __ldg(L.rp + row + 1);
  r.la = a1 - r.a0;
  r.b0 = 0;
  r.len = r.la;
  return r;
}

template <typename V>
struct TailArgs {
  int l0, L;                     // levels l0..L handled here, L = coarsest
  int ls;                        // levels ls..L run on CTA 0 alone
  int kd;                        // dense level (ls <= kd <= L) or -1: x_kd = M b_kd replaces levels kd..L
  int dn;                        // n_kd = nv_kd * d, the order of M
  int dld;                       // row stride of M: dn rounded up to a multiple of 4 (zero padding)
  int dsoff;                     // shared-memory offset (in V, 16-byte aligned) of b_kd staged for M b_kd
  const V* dm;                   // M, row-major dn x dld: the V-cycle from level kd as a matrix
  int soff[MAX_LEVELS];          // shared-memory offset (in V) of x_l, b_l, r_l for l >= ls
  TL<V> lv[MAX_LEVELS];
  CoarseArgs co;
};

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

struct ClusterSync {
  __device__ __forceinline__ void operator()() const { cluster_sync_all(); }
};
struct CtaSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// One multicolour sweep of a tail level (MODE 0: forward from zero, MODE 1:
// backward), colours separated by `sync`.  Group gg of NG handles rows
// base + gg; the entries, diagonal inverse and b of the next pass (the next
// colour's first pass at the end of a colour) are loaded before the barrier,
// since no phase of the sweep writes them; only the x gather follows it.
template <int D, int G, typename V, typename S, int MODE, bool LC, typename Sync>
__device__ __forceinline__ void tail_sweep(const TL<V>& L, int gg, int NG, int lane, Sync sync) {
  const int C = L.ncol;
  auto colour = [&](int i) { return MODE == 0 ? i : C - 1 - i; };
  RowPF<D, V, 1> cur;
  {
    const int c = colour(0), q0 = __ldg(L.cs + c), q1 = __ldg(L.cs + c + 1);
    row_prefetch<D, G, V, S, MODE, TL<V>, LC>(L, q0 + gg, q0 + gg < q1, lane, cur);
  }
  for (int i = 0; i < C; ++i) {
    const int c = colour(i), r0 = __ldg(L.cs + c), r1 = __ldg(L.cs + c + 1);
    for (int base = r0; base < r1; base += NG) {
      RowPF<D, V, 1> nxt;
      bool have = false;
      if (base + NG < r1) {
        row_prefetch<D, G, V, S, MODE, TL<V>, LC>(L, base + NG + gg, base + NG + gg < r1, lane, nxt);
        have = true;
      } else if (i + 1 < C) {
        const int c2 = colour(i + 1), q0 = __ldg(L.cs + c2), q1 = __ldg(L.cs + c2 + 1);
        row_prefetch<D, G, V, S, MODE, TL<V>, LC>(L, q0 + gg, q0 + gg < q1, lane, nxt);
        have = true;
      }
      row_finish<D, G, V, S, MODE, TL<V>, LC>(L, base + gg, base + gg < r1, lane, cur);
      if (have) cur = nxt;
    }
    sync();
  }
}

// Level l of the one-CTA part with its vectors in shared memory: x, b, r of
// level l at sm + soff[l] (n_l entries each, in that order).
template <int D, typename V>
__device__ __forceinline__ TL<V> shared_level(const TailArgs<V>& A, int l, V* sm) {
  TL<V> L = A.lv[l];
  L.x = sm + A.soff[l];
  L.b = L.x + (long long)A.lv[l].nv * D;
  L.r = L.b + (long long)A.lv[l].nv * D;
  if (l < A.L) {
    L.xc = sm + A.soff[l + 1];
    L.bc = sm + A.soff[l + 1] + (long long)A.lv[l + 1].nv * D;
  }
  return L;
}

// Levels lfrom..lto-1 of the one-CTA part, going down: forward sweep from
// zero, residual, restriction into level l+1's b; every vector in shared
// memory, the operators read through L1.
template <int D, typename V, typename S>
__device__ __forceinline__ void one_cta_down(const TailArgs<V>& A, V* sm, int lfrom, int lto) {
  constexpr int G = tail_g<D>();
  const int ng = blockDim.x / G, g = (int)threadIdx.x / G, lane = threadIdx.x & (G - 1);
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int l = lfrom; l < lto; ++l) {
    const TL<V> L = shared_level<D, V>(A, l, sm);
    tail_sweep<D, G, V, S, 0, true>(L, g, ng, lane, CtaSync());
    for (int base = 0; base < L.nv; base += ng)
      row_pass<D, G, V, S, 2, TL<V>, true>(L, base + g, base + g < L.nv, lane);
    __syncthreads();
    for (int I = tid; I < L.nvc; I += NT) restrict_row<D, V, TL<V>, true>(L, I);
    __syncthreads();
  }
}

// Levels lfrom-1 down to lto of the one-CTA part, going up: prolongation and
// correction from level l+1's x, then the backward sweep.
template <int D, typename V, typename S>
__device__ __forceinline__ void one_cta_up(const TailArgs<V>& A, V* sm, int lfrom, int lto) {
  constexpr int G = tail_g<D>();
  const int ng = blockDim.x / G, g = (int)threadIdx.x / G, lane = threadIdx.x & (G - 1);
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int l = lfrom - 1; l >= lto; --l) {
    const TL<V> L = shared_level<D, V>(A, l, sm);
    for (int i = tid; i < L.nv; i += NT) prolong_row<D, V, TL<V>, true>(L, i);
    __syncthreads();
    tail_sweep<D, G, V, S, 1, true>(L, g, ng, lane, CtaSync());
  }
}

// Levels ls..L of the V-cycle on one CTA: phases separated by CTA barriers,
// only b_ls comes in and x_ls goes out.
template <int D, typename V, typename S>
__device__ void tail_one_cta(const TailArgs<V>& A) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  V* sm = reinterpret_cast<V*>(tail_smem);
  const int tid = threadIdx.x, NT = blockDim.x;
  const int ls = A.ls, Lc = A.L;
  {
    const TL<V> Ls = shared_level<D, V>(A, ls, sm);
    for (int t = tid; t < A.lv[ls].nv * D; t += NT) Ls.b[t] = __ldcg(A.lv[ls].b + t);
  }
  __syncthreads();
  one_cta_down<D, V, S>(A, sm, ls, Lc);
  {
    const TL<V> Lcs = shared_level<D, V>(A, Lc, sm);
    if (threadIdx.x < 32) coarse_solve_warp<V, true>(A.co, Lcs.b, Lcs.x);
  }
  __syncthreads();
  one_cta_up<D, V, S>(A, sm, Lc, ls);
  {
    const TL<V> Ls = shared_level<D, V>(A, ls, sm);
    for (int t = tid; t < A.lv[ls].nv * D; t += NT) __stcg(A.lv[ls].x + t, Ls.x[t]);
  }
}

// x_kd = M b_kd on every CTA of the cluster (FP32): each CTA stages b_kd
// (global, written before the cluster barrier) in shared memory, zero-padded
// to the row stride; then one warp per row of M, lanes over 16-byte column
// groups, four partial sums, a shuffle sum, the row's x to global.
__device__ __forceinline__ void dense_level_rows(const TailArgs<float>& A, float* sb, int rank, int nct) {
  const int n = A.dn, ld = A.dld;
  const float* b = A.lv[A.kd].b;
  float* x = A.lv[A.kd].x;
  for (int t = threadIdx.x; t < ld; t += blockDim.x) sb[t] = t < n ? __ldcg(b + t) : 0.0f;
  __syncthreads();
  const float4* sb4 = reinterpret_cast<const float4*>(sb);
  const int wpc = blockDim.x >> 5, lane = threadIdx.x & 31;
  const int nw = nct * wpc, ld4 = ld >> 2;
  for (int t = rank * wpc + ((int)threadIdx.x >> 5); t < n; t += nw) {
    const float4* m4 = reinterpret_cast<const float4*>(A.dm + (long long)t * ld);
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll 4
    for (int j = lane; j < ld4; j += 32) {
      const float4 mv = __ldg(m4 + j), bv = sb4[j];
      a0 += mv.x * bv.x;
      a1 += mv.y * bv.y;
      a2 += mv.z * bv.z;
      a3 += mv.w * bv.w;
    }
    float acc = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) __stcg(x + t, acc);
  }
}

// The one-CTA part with a dense level kd: levels ls..kd-1 on CTA 0, then
// x_kd = M b_kd on the whole cluster, then back up on CTA 0.  b_kd and x_kd
// pass between the CTAs through global memory across cluster barriers.
template <int D, typename V, typename S>
__device__ void tail_dense_part(const TailArgs<V>& A, int rank, int nct) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  V* sm = reinterpret_cast<V*>(tail_smem);
  const int ls = A.ls, kd = A.kd, n_ls = A.lv[ls].nv * D, n_kd = A.dn;
  if (rank == 0 && kd > ls) {
    const TL<V> Ls = shared_level<D, V>(A, ls, sm);
    for (int t = threadIdx.x; t < n_ls; t += blockDim.x) Ls.b[t] = __ldcg(A.lv[ls].b + t);
    __syncthreads();
    one_cta_down<D, V, S>(A, sm, ls, kd);
    const TL<V> Lk = shared_level<D, V>(A, kd, sm);
    for (int t = threadIdx.x; t < n_kd; t += blockDim.x) __stcg(A.lv[kd].b + t, Lk.b[t]);
  }
  cluster_sync_all();
  dense_level_rows(A, sm + A.dsoff, rank, nct);
  cluster_sync_all();
  if (rank == 0 && kd > ls) {
    const TL<V> Lk = shared_level<D, V>(A, kd, sm);
    for (int t = threadIdx.x; t < n_kd; t += blockDim.x) Lk.x[t] = __ldcg(A.lv[kd].x + t);
    __syncthreads();
    one_cta_up<D, V, S>(A, sm, kd, ls);
    const TL<V> Ls = shared_level<D, V>(A, ls, sm);
    for (int t = threadIdx.x; t < n_ls; t += blockDim.x) __stcg(A.lv[ls].x + t, Ls.x[t]);
  }
}

// The V-cycle of all small levels in one cluster of CTAs, phases separated by
// hardware cluster barriers; every group runs the same number of loop trips
// so the sub-warp shuffles stay converged.  The smallest levels (ls..L) run
// on CTA 0 alone between two cluster barriers.
template <int D, typename V, typename S>
__device__ __forceinline__ void tail_run(const TailArgs<V>& A) {
  constexpr int G = tail_g<D>();
  const int nct = (int)cluster_size(), rank = (int)cluster_rank();
  const int ng = blockDim.x / G;
  const int gg = rank * ng + (int)threadIdx.x / G, NG = nct * ng;
  const int lane = threadIdx.x & (G - 1);
  const int tid = rank * blockDim.x + threadIdx.x, NT = nct * blockDim.x;
  const int l0 = A.l0, ls = A.ls;
  for (int l = l0; l < ls; ++l) {
    const TL<V>& L = A.lv[l];
    tail_sweep<D, G, V, S, 0, false>(L, gg, NG, lane, ClusterSync());
    for (int base = 0; base < L.nv; base += NG) row_pass<D, G, V, S, 2>(L, base + gg, base + gg < L.nv, lane);
    cluster_sync_all();
    for (int I = tid; I < L.nvc; I += NT) restrict_row<D, V>(L, I);
    cluster_sync_all();
  }
  if constexpr (std::is_same<V, float>::value) {
    if (A.kd >= 0)
      tail_dense_part<D, V, S>(A, rank, nct);
    else if (rank == 0)
      tail_one_cta<D, V, S>(A);
  } else {
    if (rank == 0) tail_one_cta<D, V, S>(A);
  }
  cluster_sync_all();
  for (int l = ls - 1; l >= l0; --l) {
    const TL<V>& L = A.lv[l];
    for (int i = tid; i < L.nv; i += NT) prolong_row<D, V>(L, i);
    cluster_sync_all();
    tail_sweep<D, G, V, S, 1, false>(L, gg, NG, lane, ClusterSync());
  }
}

template <int D, typename V, typename S>
__global__ void __launch_bounds__(TAIL_THREADS) tail_kernel(const __grid_constant__ TailArgs<V> A) {
  tail_run<D, V, S>(A);
}

// The dense level's matrix, column by column: CTA j runs the one-CTA V-cycle
// from level kd (= A.ls) on the unit vector e_j, with its own coarse-solve
// scratch, and writes the result to column j of M (row-major, n x n).
template <int D, typename V, typename S>
__global__ void __launch_bounds__(TAIL_THREADS) dense_level_kernel(const __grid_constant__ TailArgs<V> A, V* M,
                                                                   double* yscratch) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  V* sm = reinterpret_cast<V*>(tail_smem);
  const int kd = A.ls, Lc = A.L, n = A.dn, ld = A.dld, j = blockIdx.x;
  const TL<V> Lk = shared_level<D, V>(A, kd, sm);
  for (int t = threadIdx.x; t < n; t += blockDim.x) Lk.b[t] = t == j ? V(1) : V(0);
  __syncthreads();
  one_cta_down<D, V, S>(A, sm, kd, Lc);
  {
    CoarseArgs co = A.co;
    co.y = yscratch + (long long)j * co.n;
    const TL<V> Lcs = shared_level<D, V>(A, Lc, sm);
    if (threadIdx.x < 32) coarse_solve_warp<V, true>(co, Lcs.b, Lcs.x);
  }
  __syncthreads();
  one_cta_up<D, V, S>(A, sm, Lc, kd);
  for (int t = threadIdx.x; t < n; t += blockDim.x) M[(long long)t * ld + j] = Lk.x[t];
}

// ------------------------------------------------------------------ outer CG (FP64)

struct CGArgs {
  int nv;
  const int* perm;         // solve index -> input vertex
  const uint8_t* isdir;    // input dof order
  const double* lift;      // input dof order
  const double* udir;
  double* U;
  double* r;
  double* p;
  double* q;
  double* part;            // partial sums [gridDim]
  double* hist;            // relative residual history [max_iters]
  Scalars* sc;
  unsigned long long cond; // cudaGraphConditionalHandle (0 = none)
  // SELL-32 level-0 operator (diagonal block included)
  long long sell_n;        // padded rows (multiple of 32)
  long long sell_tot;      // stored entries (plane stride)
  const int* sell_rows;    // SELL position -> solve-order row (-1 = padding row)
  const long long* sell_ptr;  // slice start [nslices]
  const int* sell_w;       // slice width
  const int* sell_ci;      // [sell_tot]
  const double* sell_v;    // planes [d*d][sell_tot]
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// Write this block's partial; returns true in the last block to finish, with
// the ordered sum of all partials in *total (thread 0).  nblocks / bid: the
// blocks taking part and this block's index among them (the grid, unless
// several reductions share one launch).
__device__ __forceinline__ bool last_block_sum(double v, double* part, unsigned int* counter, double* total,
                                               int nblocks = -1, int bid = -1) {
  __shared__ double sh[32];
  __shared__ bool is_last;
  if (nblocks < 0) nblocks = (int)gridDim.x;
  if (bid < 0) bid = (int)blockIdx.x;
  const double b = block_sum(v, sh);
  if (threadIdx.x == 0) {
    part[bid] = b;
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    is_last = (t == (unsigned)nblocks - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += __ldcg(part + i);
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) {
    *total = tot;
    *counter = 0u;
  }
  return true;
}

// COND: the kernel runs inside the WHILE graph and sets its condition.  The
// variants without it are the ones a profiler can replay.
template <bool COND>
__device__ __forceinline__ void set_cond(unsigned long long h, unsigned int v) {
  if constexpr (COND) {
    if (h) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
  }
}

// r = F - A u_D at free dofs (0 at Dirichlet dofs), gathered into solve order;
// U = p = 0; res0 = ||r||; b_0 = (V) r.
template <int D, typename V, bool COND>
__global__ void __launch_bounds__(CG_THREADS) cg_init_kernel(CGArgs a, const double* __restrict__ F, V* b0) {
  double acc = 0.0;
  const long long n = (long long)a.nv * D;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / D;
    const int c = (int)(t - r * D);
    const long long g = (long long)__ldg(a.perm + r) * D + c;
    const double v = __ldg(a.isdir + g) ? 0.0 : F[g] - __ldg(a.lift + g);
    a.r[t] = v;
    a.U[t] = 0.0;
    a.p[t] = 0.0;
    b0[t] = (V)v;
    acc += v * v;
  }
  double tot;
  if (last_block_sum(acc, a.part, &a.sc->cnt[0], &tot) && threadIdx.x == 0) {
    Scalars* s = a.sc;
    s->res0 = sqrt(tot);
    s->rr = tot;
    s->relres = 1.0;
    s->iter = 0;
    s->bodies = 0;
    s->first = 1;
    s->status = 0;
    s->abort = 0;
    s->done = (s->res0 == 0.0) ? 1 : 0;
    if (s->done) s->relres = 0.0;
    set_cond<COND>(a.cond, s->done ? 0u : 1u);
  }
}

// rho_new = r . z; beta = rho_new / rho (0 on the first iteration)
template <int D, typename V, bool COND>
__global__ void __launch_bounds__(CG_THREADS) rz_kernel(CGArgs a, const V* __restrict__ z) {
  double acc = 0.0;
  const long long n = (long long)a.nv * D;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    acc += a.r[t] * (double)__ldcg(z + t);
  // hard bound on loop bodies, independent of the reductions: the device-side
  // WHILE loop never runs more than max_iters + 2 bodies
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Scalars* s = a.sc;
    s->bodies += 1;
    if (s->bodies > s->max_iters + 2) {
      s->done = 1;
      s->status = VASMG_ERR_TIMEOUT;
      set_cond<COND>(a.cond, 0u);
    }
  }
  double tot;
  if (last_block_sum(acc, a.part, &a.sc->cnt[1], &tot) && threadIdx.x == 0) {
    Scalars* s = a.sc;
    s->beta = s->first ? 0.0 : tot / s->rho;
    s->rho = tot;
    s->first = 0;
  }
}

template <int D, typename V>
__global__ void __launch_bounds__(CG_THREADS) p_update_kernel(CGArgs a, const V* __restrict__ z) {
  const double beta = a.sc->beta;
  const long long n = (long long)a.nv * D;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    a.p[t] = (double)__ldcg(z + t) + beta * a.p[t];
}

// q = A p (SELL-32, one thread per row, one warp per slice), p.q, alpha.
template <int D, bool COND>
__global__ void __launch_bounds__(CG_THREADS) spmv_sell_kernel(CGArgs a, int with_dot) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nslices = a.sell_n >> 5;
  double dot = 0.0;
  for (long long s = warp; s < nslices; s += nwarps) {
    const long long base = __ldg(a.sell_ptr + s) + lane;
    const int w = __ldg(a.sell_w + s);
    const int row = __ldg(a.sell_rows + (s << 5) + lane);
    double acc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = 0.0;
    for (int k = 0; k < w; ++k) {
      const long long idx = base + ((long long)k << 5);
      const int j = __ldg(a.sell_ci + idx);
      double pj[D];
#pragma unroll
      for (int bb = 0; bb < D; ++bb) pj[bb] = a.p[(long long)j * D + bb];
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int bb = 0; bb < D; ++bb)
          acc[c] = fma(__ldg(a.sell_v + (long long)(c * D + bb) * a.sell_tot + idx), pj[bb], acc[c]);
    }
    if (row >= 0) {
#pragma unroll
      for (int c = 0; c < D; ++c) {
        a.q[(long long)row * D + c] = acc[c];
        dot = fma(acc[c], a.p[(long long)row * D + c], dot);
      }
    }
  }
  if (!with_dot) return;
  double tot;
  if (last_block_sum(dot, a.part, &a.sc->cnt[2], &tot) && threadIdx.x == 0) {
    Scalars* s = a.sc;
    s->pq = tot;
    if (!(tot > 0.0)) {
      s->status = VASMG_ERR_BREAKDOWN;
      s->done = 1;
      s->alpha = 0.0;
      set_cond<COND>(a.cond, 0u);
    } else {
      s->alpha = s->rho / tot;
    }
  }
}

// U += alpha p; r -= alpha q; ||r||; stop test; b_0 = (V) r.
template <int D, typename V, bool COND>
__global__ void __launch_bounds__(CG_THREADS) cg_update_kernel(CGArgs a, V* b0) {
  if (a.sc->done) return;  // breakdown in spmv
  const double alpha = a.sc->alpha;
  double acc = 0.0;
  const long long n = (long long)a.nv * D;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    a.U[t] += alpha * a.p[t];
    const double rv = a.r[t] - alpha * a.q[t];
    a.r[t] = rv;
    b0[t] = (V)rv;
    acc += rv * rv;
  }
  double tot;
  if (last_block_sum(acc, a.part, &a.sc->cnt[3], &tot) && threadIdx.x == 0) {
    Scalars* s = a.sc;
    s->rr = tot;
    s->relres = sqrt(tot) / s->res0;
    s->iter += 1;
    if (s->iter <= s->max_iters) a.hist[s->iter - 1] = s->relres;
    if (s->abort) {
      s->done = 1;
      s->status = VASMG_ERR_TIMEOUT;
    } else if (s->relres < s->tol) {
      s->done = 1;
      s->status = VASMG_OK;
    } else if (!(s->relres == s->relres)) {
      s->done = 1;
      s->status = VASMG_ERR_BREAKDOWN;
    } else if (s->iter >= s->max_iters) {
      s->done = 1;
      s->status = VASMG_NOT_CONVERGED;
    }
    if (s->bodies > s->max_iters + 2) s->done = 1;
    set_cond<COND>(a.cond, s->done ? 0u : 1u);
  }
}

// U (solve order) -> user order, Dirichlet values written in.
template <int D>
__global__ void cg_final_kernel(CGArgs a, double* __restrict__ Uout) {
  const long long n = (long long)a.nv * D;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / D;
    const int c = (int)(t - r * D);
    const long long g = (long long)__ldg(a.perm + r) * D + c;
    Uout[g] = __ldg(a.isdir + g) ? __ldg(a.udir + g) : a.U[t];
  }
}


// ------------------------------------------------------------------ several right-hand sides (solve_multi.cu)

// What the engine of one hierarchy hands to its solver for several
// right-hand sides: the level views (operators, transfers, region tables and
// progress words, with the single-vector x, b, r), the lanes per row of the
// region levels, the tail launch's arguments, and the outer CG's layout.  The
// device arrays stay owned by the engine; the view is taken again before
// every call, so new values (vasmg_update_data) are seen.
template <typename V>
struct EngineView {
  cudaStream_t stream = 0;
  int L = 0, lt = 0, nct = 1, sms = 1, max_iters = 1000, use_graph = 1;
  std::vector<LV<V>> lv;
  std::vector<int> G;              // lanes per row of the region levels (l < lt)
  std::vector<i64> nv;             // vertices per level
  std::vector<double> pnnz;        // transfer entries of level l -> l+1
  TailArgs<V> ta;                  // the tail launch from level lt (dense level fields set if used)
  size_t tail_smem = 0;            // its dynamic shared memory, without the staging of b_kd
  CGArgs cga;                      // level-0 FP64 operator (SELL), permutation, Dirichlet data
  int cg_blocks = 1, spmv_blocks = 1;
  i64 sell_real_entries = 0;
  int* ctr = nullptr;              // per-level launch counters (epochs), shared with the single path
  int dim = 2, device = 0;
  double* Fbuf = nullptr;          // the engine's staging of F and U (solve order / user order)
  double* Ubuf = nullptr;
  // per level, the engine's StagedOp<S> of the forward / backward sweep
  // (3D region levels whose sweeps stream a staged copy), else null
  std::vector<const void*> stg_fwd, stg_bwd;
};

// k independent PCG solves on one hierarchy whose every sweep, transfer and
// SpMV reads the operators once for all k (solve_multi.cu).
struct MultiBase {
  virtual ~MultiBase() {}
  virtual void set_view(const EngineView<float>& v) = 0;
  virtual int solve(int k, const double* const* F, double* const* U, double tol, vasmg_stats* st,
                    i64* launches) = 0;
  virtual double time(int which, int level, int k, int reps, double* bytes) = 0;
};
template <int D, typename S>
MultiBase* make_multi(const EngineView<float>& v);

// Several hierarchies advanced together, one right-hand side each: every
// region level's sweeps, residuals and transfers of all of them in one launch
// per level and phase, their tails in one launch (a cluster each), and the
// outer CG kernels of all of them in one launch each (solve_multi.cu).
// views: the engines' views (same V-cycle precision S, gamma 1, not
// additive); F[i], U[i]: host or device vectors of hierarchy i.  Each result
// is the one vasmg_solve gives for that hierarchy alone.  *launches receives
// the kernels launched.
template <typename S>
int batch_solve(const std::vector<EngineView<float>>& views, cudaStream_t stream, const double* const* F,
                double* const* U, double tol, vasmg_stats* st, i64* launches);
// CTAs of the batched region sweep that the device holds at once
template <typename S>
int batch_sweep_capacity();


}  // namespace vasmg
