// Several right-hand sides on one hierarchy: k independent PCG solves (Alg. 2
// with the V-cycle of Alg. 3 as the preconditioner) advanced together, KR at a
// time (KR in {2, 4, 8}; unused slots carry a zero right-hand side, which PCG
// finishes at its first test).
//
// Every kernel of an iteration reads the operators once for all KR vectors:
// the multicolour sweeps and residuals read each block once and apply it to
// KR gathered vertex vectors, the transfers read each weight once, the dense
// coarse level reads M once, and the FP64 SpMV reads each block once for up to
// four vectors.  The V-cycle's vectors are interleaved, entry (vertex v,
// right-hand side i, component a) at (v KR + i) D + a, so one neighbour gather
// is one contiguous KR D read.  The outer CG's vectors are stored one
// right-hand side after another.
//
// Each right-hand side's arithmetic is exactly that of vasmg_solve: the same
// lanes per row, the same order of additions within a row, the same
// reduction trees (the CG kernels keep the single solve's grid and give
// every right-hand side its own partials and counters).  So each result is
// bitwise the one vasmg_solve gives alone, with the same iteration count; a
// right-hand side that has converged keeps its iterate while the others go on.
#include <cstring>
#include <memory>

#include "solve_dev.cuh"

namespace vasmg {

constexpr int DFM_THREADS = 256;    // threads of the batched sweep CTAs and of the plain batched kernels
constexpr int TAILM_THREADS = 512;  // threads of the multi tail CTAs (more registers per thread than the single tail)
constexpr int KMAX = 8;             // right-hand sides per pass
constexpr int KG_SPMV = 4;          // right-hand sides per SpMV launch

// N consecutive vector values (a vertex's KR x D entries), through L1 on the
// region levels and from L2 on the tail's levels (see ld_shared_vec): 16-byte
// loads when N is a multiple of 4 (the block starts on a 16-byte boundary),
// else 8-byte loads.
template <int N, bool L1>
__device__ __forceinline__ void ld_vec_n(const float* p, float (&v)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
      const float4 t = ld_shared_vec<L1>(reinterpret_cast<const float4*>(p) + q);
      v[4 * q] = t.x, v[4 * q + 1] = t.y, v[4 * q + 2] = t.z, v[4 * q + 3] = t.w;
    }
  } else if constexpr (N % 2 == 0) {
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      const float2 t = ld_shared_vec<L1>(reinterpret_cast<const float2*>(p) + q);
      v[2 * q] = t.x, v[2 * q + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = ld_shared_vec<L1>(p + q);
  }
}

// ------------------------------------------------------------------ rows with KR right-hand sides

template <int D, int KR, typename V>
struct RowPFM {
  RowSeg sg;
  int cj;
  V a[D * D];
  V di[D];
};

// Loads what nothing writes during the sweep: the row range, this lane's
// first entry and the diagonal inverse row (b of the right-hand sides is
// loaded when the row is finished, which keeps the prefetched state small).
template <int D, int KR, typename V, typename S, int MODE, typename L_t>
__device__ __forceinline__ void rowm_prefetch(const L_t& L, int row, bool valid, int lane, RowPFM<D, KR, V>& st) {
  st.sg = RowSeg{0, 0, 0, 0};
  if (valid) st.sg = seg_range<MODE>(L, row);
  const int* ciA;
  const S* offA;
  long long nA;
  const int* ciB;
  const S* offB;
  long long nB;
  seg_ptrs<MODE, S>(L, ciA, offA, nA, ciB, offB, nB);
  st.cj = -1;
  if (lane < st.sg.len) st.cj = seg_entry<D, V, S>(st.sg, lane, ciA, offA, nA, ciB, offB, nB, st.a);
  if (MODE != 2 && valid && lane < D) {
#pragma unroll
    for (int bb = 0; bb < D; ++bb) st.di[bb] = __ldg((const V*)L.dinv + (long long)(lane * D + bb) * L.nv + row);
  }
}

// The row's products for every right-hand side, G lanes over its entries in
// the order e = lane, lane + G, ... (as the single sweep), the lanes' sums
// combined by the same shuffle tree; lanes a < D then write component a.
template <int D, int KR, typename V, typename S, int MODE, typename L_t>
__device__ __forceinline__ void rowm_finish(const L_t& L, int row, bool valid, int lane, int G,
                                            const RowPFM<D, KR, V>& st) {
  V acc[KR][D];
#pragma unroll
  for (int i = 0; i < KR; ++i)
#pragma unroll
    for (int a = 0; a < D; ++a) acc[i][a] = V(0);
  // b of every right-hand side (lanes a < D write the row), in flight while the entries are gathered
  V bv[KR * D];
  if (MODE != 2 && valid && lane < D) ld_vec_n<KR * D, false>((const V*)L.b + (long long)row * KR * D, bv);
  if (st.cj >= 0) {
    V xj[KR * D];
    ld_vec_n<KR * D, gather_l1<L_t, false>()>((const V*)L.x + (long long)st.cj * KR * D, xj);
#pragma unroll
    for (int i = 0; i < KR; ++i)
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int bb = 0; bb < D; ++bb) acc[i][a] += st.a[a * D + bb] * xj[i * D + bb];
  }
  const int* ciA;
  const S* offA;
  long long nA;
  const int* ciB;
  const S* offB;
  long long nB;
  seg_ptrs<MODE, S>(L, ciA, offA, nA, ciB, offB, nB);
  for (int e = lane + G; e < st.sg.len; e += G) {
    V blk[D * D];
    const int j = seg_entry<D, V, S>(st.sg, e, ciA, offA, nA, ciB, offB, nB, blk);
    V xj[KR * D];
    ld_vec_n<KR * D, gather_l1<L_t, false>()>((const V*)L.x + (long long)j * KR * D, xj);
#pragma unroll
    for (int i = 0; i < KR; ++i)
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int bb = 0; bb < D; ++bb) acc[i][a] += blk[a * D + bb] * xj[i * D + bb];
  }
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < KR; ++i)
#pragma unroll
      for (int a = 0; a < D; ++a) acc[i][a] += __shfl_xor_sync(0xffffffffu, acc[i][a], o, G);
  if (!valid || lane >= D) return;
#pragma unroll
  for (int i = 0; i < KR; ++i) {
    if (MODE == 2) {
      V v = acc[i][0];
#pragma unroll
      for (int a = 1; a < D; ++a)
        if (lane == a) v = acc[i][a];
      __stcg((V*)L.r + ((long long)row * KR + i) * D + lane, -v);
    } else {
      V s = V(0);
#pragma unroll
      for (int bb = 0; bb < D; ++bb) s += st.di[bb] * (bv[i * D + bb] - acc[i][bb]);
      __stcg((V*)L.x + ((long long)row * KR + i) * D + lane, s);
    }
  }
}

template <int D, int KR, typename V, typename S, int MODE>
__device__ __forceinline__ void rowsm_pipelined(const LV<V>& L, int r0, int r1, int G, RowPFM<D, KR, V>& cur) {
  const int NG = (int)blockDim.x / G;
  const int g = threadIdx.x / G, lane = threadIdx.x & (G - 1);
  for (int base = r0; base < r1; base += NG) {
    const int nb = base + NG;
    RowPFM<D, KR, V> nxt;
    if (nb < r1) rowm_prefetch<D, KR, V, S, MODE>(L, nb + g, nb + g < r1, lane, nxt);
    rowm_finish<D, KR, V, S, MODE>(L, base + g, base + g < r1, lane, G, cur);
    if (nb < r1) cur = nxt;
  }
}

// b_{l+1} = R r_l for coarse row I (one thread), every right-hand side.
template <int D, int KR, typename V, typename L_t>
__device__ __forceinline__ void restrictm_row(const L_t& L, int I) {
  V acc[KR * D];
#pragma unroll
  for (int q = 0; q < KR * D; ++q) acc[q] = V(0);
  for (int t = __ldg(L.rrp + I); t < __ldg(L.rrp + I + 1); ++t) {
    const int i = __ldg(L.rci + t);
    const V w = __ldg((const V*)L.rw + t);
    V ri[KR * D];
    ld_vec_n<KR * D, gather_l1<L_t, false>()>((const V*)L.r + (long long)i * KR * D, ri);
#pragma unroll
    for (int q = 0; q < KR * D; ++q) acc[q] += w * ri[q];
  }
#pragma unroll
  for (int q = 0; q < KR * D; ++q) __stcg((V*)L.bc + (long long)I * KR * D + q, acc[q]);
}

// x_l += P x_{l+1} for fine row i (one thread), masked at dead dofs.
template <int D, int KR, typename V, typename L_t>
__device__ __forceinline__ void prolongm_row(const L_t& L, int i) {
  V acc[KR * D];
#pragma unroll
  for (int q = 0; q < KR * D; ++q) acc[q] = V(0);
  for (int t = __ldg(L.prp + i); t < __ldg(L.prp + i + 1); ++t) {
    const int J = __ldg(L.pci + t);
    const V w = __ldg((const V*)L.pw + t);
    V xJ[KR * D];
    ld_vec_n<KR * D, gather_l1<L_t, false>()>((const V*)L.xc + (long long)J * KR * D, xJ);
#pragma unroll
    for (int q = 0; q < KR * D; ++q) acc[q] += w * xJ[q];
  }
  const uint8_t dm = __ldg(L.dead + i);
#pragma unroll
  for (int k = 0; k < KR; ++k)
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (!((dm >> a) & 1)) {
        V* px = (V*)L.x + ((long long)i * KR + k) * D + a;
        __stcg(px, __ldcg((const V*)px) + acc[k * D + a]);
      }
}

// ------------------------------------------------------------------ region launches

// The multi sweeps hold as many CTAs per SM as the single sweeps' regions
// need: 2D levels with FP32 vectors have one 1024-thread region per SM (their
// multi CTAs take 512 threads, as many as the registers of 8 right-hand
// sides allow), 3D levels two 256-thread regions.
template <int D, typename V>
constexpr int dfm_threads() { return (D == 2 && sizeof(V) == 4) ? 512 : 256; }
template <int D, typename V>
constexpr int dfm_min_blocks() { return df_min_blocks<D, V>(); }

// Forward sweep from zero of one region level, KR right-hand sides (the waits
// and stages of vdown_kernel).
template <int D, int KR, typename V, typename S>
__global__ void __launch_bounds__(dfm_threads<D, V>(), dfm_min_blocks<D, V>())
    vdownm_kernel(const __grid_constant__ LV<V> L, Scalars* sc, int G) {
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
      RowPFM<D, KR, V> cur;
      rowm_prefetch<D, KR, V, S, 0>(L, r0 + g, r0 + g < r1, lane, cur);
      if (c > 0 && !wait_regions(L.nb + nb0, nnb, L.pg_d, epoch, (unsigned)c, abort_flag)) break;
      rowsm_pipelined<D, KR, V, S, 0>(L, r0, r1, G, cur);
    }
    publish_stage(mine, epoch, (unsigned)(c + 1));
  }
  leave(L.ctr, C_DEXIT, C_DEPOCH);
}

// Backward sweep of one region level, KR right-hand sides.
template <int D, int KR, typename V, typename S>
__global__ void __launch_bounds__(dfm_threads<D, V>(), dfm_min_blocks<D, V>())
    vupm_kernel(const __grid_constant__ LV<V> L, Scalars* sc, int G) {
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
      RowPFM<D, KR, V> cur;
      rowm_prefetch<D, KR, V, S, 1>(L, r0 + g, r0 + g < r1, lane, cur);
      if (stage > 0 && !wait_regions(L.nb + nb0, nnb, L.pg_u, epoch, stage, abort_flag)) break;
      rowsm_pipelined<D, KR, V, S, 1>(L, r0, r1, G, cur);
    }
    publish_stage(mine, epoch, ++stage);
  }
  leave(L.ctr, C_UEXIT, C_UEPOCH);
}

template <int D, int KR, typename V, typename S>
__global__ void __launch_bounds__(256) residualm_kernel(const __grid_constant__ LV<V> L, int G) {
  const int NG = 256 / G;
  const int g = threadIdx.x / G, lane = threadIdx.x & (G - 1);
  for (int base = blockIdx.x * NG; base < L.nv; base += gridDim.x * NG) {
    RowPFM<D, KR, V> st;
    rowm_prefetch<D, KR, V, S, 2>(L, base + g, base + g < L.nv, lane, st);
    rowm_finish<D, KR, V, S, 2>(L, base + g, base + g < L.nv, lane, G, st);
  }
}

template <int D, int KR, typename V>
__global__ void __launch_bounds__(256) restrictm_kernel(const __grid_constant__ LV<V> L) {
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < L.nvc; I += gridDim.x * blockDim.x)
    restrictm_row<D, KR, V>(L, I);
}

template <int D, int KR, typename V>
__global__ void __launch_bounds__(256) prolongm_kernel(const __grid_constant__ LV<V> L) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.nv; i += gridDim.x * blockDim.x)
    prolongm_row<D, KR, V>(L, i);
}

// ------------------------------------------------------------------ staged region sweeps (3D), KR right-hand sides

// The consumers of vstaged_kernel with KR right-hand sides: the same chunks of
// the level's staged copy (the producer is stg_produce), each slot applied to
// the KR interleaved vectors of its column, each right-hand side's sums in the
// order of rowm_finish.  b of a row is loaded when its group starts the row.
template <int D, int KR, typename V, typename S, int MODE>
__device__ __forceinline__ void stgm_consume(const LV<V>& L, const StagedOp<S>& O, int k, int R, int C,
                                             unsigned epoch, unsigned long long* full, unsigned long long* empty,
                                             const unsigned char* ring, int* abort_flag, int G) {
  constexpr int NS = stg_stages<S>(), CB = stg_chunk_bytes<S>(), EPT = stg_ept<S>(), N = KR * D;
  const int NG = STG_T / G;
  const int tid = threadIdx.x, g = tid / G, lane = tid & (G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((tid & 31) & ~(G - 1)));
  const int nb0 = __ldg(L.nb_rp + k), nnb = __ldg(L.nb_rp + k + 1) - nb0;
  unsigned long long* pg = MODE == 0 ? L.pg_d : L.pg_u;
  long long q = 0;  // chunks taken
  for (int i = 0; i < C; ++i) {
    const int c = MODE == 0 ? i : C - 1 - i;
    const int r0 = __ldg(L.RS + c * (R + 1) + k), r1 = __ldg(L.RS + c * (R + 1) + k + 1);
    if (r0 < r1) {
      const int step = c * R + k;
      int j = r0 + __ldg(O.goff + (long long)step * (NG + 1) + g);
      const int j1 = r0 + __ldg(O.goff + (long long)step * (NG + 1) + g + 1);
      int row = j < j1 ? __ldg(O.srow + j) : -1;
      int rown = j + 1 < j1 ? __ldg(O.srow + j + 1) : -1;
      V di[D], bv[N];
      auto row_data = [&]() {
        if (row >= 0 && lane < D) {
#pragma unroll
          for (int bb = 0; bb < D; ++bb) di[bb] = __ldg((const V*)L.dinv + (long long)(lane * D + bb) * L.nv + row);
          ld_vec_n<N, false>((const V*)L.b + (long long)row * N, bv);
        }
      };
      row_data();
      if (i > 0 && !wait_regions<STG_T>(L.nb + nb0, nnb, pg, epoch, (unsigned)i, abort_flag)) break;
      const int nact = __ldg(O.step_nact + step), ne = EPT * nact;
      const long long nch = (__ldg(O.step_off + step + 1) - __ldg(O.step_off + step)) / ne;
      V acc[KR][D];
#pragma unroll
      for (int r = 0; r < KR; ++r)
#pragma unroll
        for (int a = 0; a < D; ++a) acc[r][a] = V(0);
      for (long long t = 0; t < nch; ++t, ++q) {
        const int s = (int)(q % NS);
        // warp-uniform: a lane group never splits between taking and skipping a chunk
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[s], (unsigned)((q / NS) & 1), abort_flag));
        const unsigned char* chunk = ring + s * CB;
        // up to 4 right-hand sides, two slots at a time with their gathers in
        // flight together; 8 right-hand sides one slot at a time (registers)
        if constexpr (KR > 4) {
#pragma unroll
        for (int h = 0; h < EPT; ++h) {
          const int v = ok && tid < nact ? reinterpret_cast<const int*>(chunk)[h * nact + tid] : -1;
          if (v < 0) continue;
          const int col = v & STG_NONE;
          if (col != STG_NONE) {
            V xj[N];
            ld_vec_n<N, true>((const V*)L.x + (long long)col * N, xj);
            V blk[9];
            stg_block<V, S>(chunk, ne, h * nact + tid, blk);
#pragma unroll
            for (int r = 0; r < KR; ++r)
#pragma unroll
              for (int a = 0; a < D; ++a)
#pragma unroll
                for (int bb = 0; bb < D; ++bb) acc[r][a] += blk[a * D + bb] * xj[r * D + bb];
          }
          if (v & STG_END) {
            // the row is done: the group's sums, x_row of every right-hand side, the next row
            for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
              for (int r = 0; r < KR; ++r)
#pragma unroll
                for (int a = 0; a < D; ++a) acc[r][a] += __shfl_xor_sync(gmask, acc[r][a], o, G);
            if (row >= 0 && lane < D) {
#pragma unroll
              for (int r = 0; r < KR; ++r) {
                V sum = V(0);
#pragma unroll
                for (int bb = 0; bb < D; ++bb) sum += di[bb] * (bv[r * D + bb] - acc[r][bb]);
                __stcg((V*)L.x + ((long long)row * KR + r) * D + lane, sum);
              }
            }
#pragma unroll
            for (int r = 0; r < KR; ++r)
#pragma unroll
              for (int a = 0; a < D; ++a) acc[r][a] = V(0);
            ++j;
            row = rown;
            rown = j + 1 < j1 ? __ldg(O.srow + j + 1) : -1;
            row_data();
          }
        }
        } else {
        constexpr int PK = 2;
#pragma unroll
        for (int h0 = 0; h0 < EPT; h0 += PK) {
          int vv[PK];
          V xj[PK][N];
#pragma unroll
          for (int u = 0; u < PK; ++u) {
            vv[u] = ok && tid < nact ? reinterpret_cast<const int*>(chunk)[(h0 + u) * nact + tid] : -1;
            const int col = vv[u] & STG_NONE;
            if (vv[u] >= 0 && col != STG_NONE) ld_vec_n<N, true>((const V*)L.x + (long long)col * N, xj[u]);
          }
#pragma unroll
          for (int u = 0; u < PK; ++u) {
          const int v = vv[u], h = h0 + u;
          if (v < 0) continue;
          const int col = v & STG_NONE;
          if (col != STG_NONE) {
            V blk[9];
            stg_block<V, S>(chunk, ne, h * nact + tid, blk);
#pragma unroll
            for (int r = 0; r < KR; ++r)
#pragma unroll
              for (int a = 0; a < D; ++a)
#pragma unroll
                for (int bb = 0; bb < D; ++bb) acc[r][a] += blk[a * D + bb] * xj[u][r * D + bb];
          }
          if (v & STG_END) {
            // the row is done: the group's sums, x_row of every right-hand side, the next row
            for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
              for (int r = 0; r < KR; ++r)
#pragma unroll
                for (int a = 0; a < D; ++a) acc[r][a] += __shfl_xor_sync(gmask, acc[r][a], o, G);
            if (row >= 0 && lane < D) {
#pragma unroll
              for (int r = 0; r < KR; ++r) {
                V sum = V(0);
#pragma unroll
                for (int bb = 0; bb < D; ++bb) sum += di[bb] * (bv[r * D + bb] - acc[r][bb]);
                __stcg((V*)L.x + ((long long)row * KR + r) * D + lane, sum);
              }
            }
#pragma unroll
            for (int r = 0; r < KR; ++r)
#pragma unroll
              for (int a = 0; a < D; ++a) acc[r][a] = V(0);
            ++j;
            row = rown;
            rown = j + 1 < j1 ? __ldg(O.srow + j + 1) : -1;
            row_data();
          }
          }
        }
        }
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[s]);
      }
    }
    publish_stage<STG_T>(pg + k, epoch, (unsigned)(i + 1));
  }
}

// Forward sweep from zero (MODE 0) or backward sweep (MODE 1) of a 3D region
// level with KR right-hand sides, reading the level's staged copy (as
// vstaged_kernel; G lanes per row, a runtime argument).
template <int D, int KR, typename V, typename S, int MODE>
__global__ void __launch_bounds__(STG_T + 32, 2)
    vstagedm_kernel(const __grid_constant__ LV<V> L, const __grid_constant__ StagedOp<S> O, Scalars* sc, int G) {
  static_assert(D == 3, "the staged layout holds 3 x 3 blocks");
  constexpr int NS = stg_stages<S>();
  extern __shared__ __align__(128) unsigned char stgm_ring[];
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
    if (threadIdx.x == STG_T) stg_produce<S, MODE, true>(O, k, L.R, L.ncol, full, empty, stgm_ring, abort_flag);
  } else {
    stgm_consume<D, KR, V, S, MODE>(L, O, k, L.R, L.ncol, epoch, full, empty, stgm_ring, abort_flag, G);
  }
  leave(L.ctr, MODE == 0 ? C_DEXIT : C_UEXIT, MODE == 0 ? C_DEPOCH : C_UEPOCH);
}

// ------------------------------------------------------------------ tail

// One multicolour sweep of a tail level on the cluster, KR right-hand sides.
template <int D, int KR, typename V, typename S, int MODE>
__device__ __forceinline__ void tailm_sweep(const TL<V>& L, int gg, int NG, int lane, int G) {
  const int C = L.ncol;
  auto colour = [&](int i) { return MODE == 0 ? i : C - 1 - i; };
  RowPFM<D, KR, V> cur;
  {
    const int c = colour(0), q0 = __ldg(L.cs + c), q1 = __ldg(L.cs + c + 1);
    rowm_prefetch<D, KR, V, S, MODE>(L, q0 + gg, q0 + gg < q1, lane, cur);
  }
  for (int i = 0; i < C; ++i) {
    const int c = colour(i), r0 = __ldg(L.cs + c), r1 = __ldg(L.cs + c + 1);
    for (int base = r0; base < r1; base += NG) {
      RowPFM<D, KR, V> nxt;
      bool have = false;
      if (base + NG < r1) {
        rowm_prefetch<D, KR, V, S, MODE>(L, base + NG + gg, base + NG + gg < r1, lane, nxt);
        have = true;
      } else if (i + 1 < C) {
        const int c2 = colour(i + 1), q0 = __ldg(L.cs + c2), q1 = __ldg(L.cs + c2 + 1);
        rowm_prefetch<D, KR, V, S, MODE>(L, q0 + gg, q0 + gg < q1, lane, nxt);
        have = true;
      }
      rowm_finish<D, KR, V, S, MODE>(L, base + gg, base + gg < r1, lane, G, cur);
      if (have) cur = nxt;
    }
    cluster_sync_all();
  }
}

// Entry t of a level's vector of right-hand side i in the interleaved layout.
template <int D, int KR>
__device__ __forceinline__ long long mix(long long t, int i) {
  return ((t / D) * KR + i) * D + (t % D);
}

// Levels ls..L of the V-cycle on CTA 0 for right-hand side i, with the
// single solve's code (vectors in shared memory): b_ls of right-hand side i
// comes in, its x_ls goes out.
template <int D, int KR, typename V, typename S>
__device__ void tailm_one_cta(const TailArgs<V>& A, int i) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  V* sm = reinterpret_cast<V*>(tail_smem);
  const int tid = threadIdx.x, NT = blockDim.x;
  const int ls = A.ls, Lc = A.L, n_ls = A.lv[ls].nv * D;
  {
    const TL<V> Ls = shared_level<D, V>(A, ls, sm);
    for (int t = tid; t < n_ls; t += NT) Ls.b[t] = __ldcg(A.lv[ls].b + mix<D, KR>(t, i));
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
    for (int t = tid; t < n_ls; t += NT) __stcg(A.lv[ls].x + mix<D, KR>(t, i), Ls.x[t]);
  }
  __syncthreads();
}

// x_kd = M b_kd for every right-hand side on every CTA of the cluster: b_kd of
// each right-hand side staged in shared memory (zero-padded to the row
// stride), one warp per row of M; every right-hand side's sums are formed as
// in dense_level_rows.
template <int D, int KR>
__device__ __forceinline__ void dense_rows_m(const TailArgs<float>& A, float* sb, int rank, int nct) {
  const int n = A.dn, ld = A.dld, ld4 = ld >> 2;
  const float* b = A.lv[A.kd].b;
  float* x = A.lv[A.kd].x;
  for (int t = threadIdx.x; t < KR * ld; t += blockDim.x) {
    const int i = t / ld, c = t - i * ld;
    sb[t] = c < n ? __ldcg(b + mix<D, KR>(c, i)) : 0.0f;
  }
  __syncthreads();
  const float4* sb4 = reinterpret_cast<const float4*>(sb);
  const int wpc = blockDim.x >> 5, lane = threadIdx.x & 31;
  const int nw = nct * wpc;
  for (int t = rank * wpc + ((int)threadIdx.x >> 5); t < n; t += nw) {
    const float4* m4 = reinterpret_cast<const float4*>(A.dm + (long long)t * ld);
    float a[KR][4];
#pragma unroll
    for (int i = 0; i < KR; ++i) a[i][0] = a[i][1] = a[i][2] = a[i][3] = 0.0f;
    for (int j = lane; j < ld4; j += 32) {
      const float4 mv = __ldg(m4 + j);
#pragma unroll
      for (int i = 0; i < KR; ++i) {
        const float4 bv = sb4[i * ld4 + j];
        a[i][0] += mv.x * bv.x;
        a[i][1] += mv.y * bv.y;
        a[i][2] += mv.z * bv.z;
        a[i][3] += mv.w * bv.w;
      }
    }
#pragma unroll
    for (int i = 0; i < KR; ++i) {
      float acc = (a[i][0] + a[i][1]) + (a[i][2] + a[i][3]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) __stcg(x + mix<D, KR>(t, i), acc);
    }
  }
}

// The one-CTA part with a dense level kd (FP32): levels ls..kd-1 on CTA 0 for
// each right-hand side in turn (their shared vectors saved to `stash` for the
// way up), x_kd = M b_kd for all of them on the cluster, then back up on CTA
// 0 one right-hand side at a time.
template <int D, int KR, typename S>
__device__ void tailm_dense_part(const TailArgs<float>& A, int rank, int nct, float* stash) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  float* sm = reinterpret_cast<float*>(tail_smem);
  const int ls = A.ls, kd = A.kd, n_ls = A.lv[ls].nv * D, n_kd = A.dn;
  const int s0 = A.soff[ls], s1 = A.soff[kd], slen = s1 - s0;
  if (rank == 0 && kd > ls) {
    for (int i = 0; i < KR; ++i) {
      const TL<float> Ls = shared_level<D, float>(A, ls, sm);
      for (int t = threadIdx.x; t < n_ls; t += blockDim.x) Ls.b[t] = __ldcg(A.lv[ls].b + mix<D, KR>(t, i));
      __syncthreads();
      one_cta_down<D, float, S>(A, sm, ls, kd);
      const TL<float> Lk = shared_level<D, float>(A, kd, sm);
      for (int t = threadIdx.x; t < n_kd; t += blockDim.x) __stcg(A.lv[kd].b + mix<D, KR>(t, i), Lk.b[t]);
      for (int t = threadIdx.x; t < slen; t += blockDim.x) stash[(long long)i * slen + t] = sm[s0 + t];
      __syncthreads();
    }
  }
  cluster_sync_all();
  dense_rows_m<D, KR>(A, sm + A.dsoff, rank, nct);
  cluster_sync_all();
  if (rank == 0 && kd > ls) {
    for (int i = 0; i < KR; ++i) {
      for (int t = threadIdx.x; t < slen; t += blockDim.x) sm[s0 + t] = stash[(long long)i * slen + t];
      const TL<float> Lk = shared_level<D, float>(A, kd, sm);
      for (int t = threadIdx.x; t < n_kd; t += blockDim.x) Lk.x[t] = __ldcg(A.lv[kd].x + mix<D, KR>(t, i));
      __syncthreads();
      one_cta_up<D, float, S>(A, sm, kd, ls);
      const TL<float> Ls = shared_level<D, float>(A, ls, sm);
      for (int t = threadIdx.x; t < n_ls; t += blockDim.x) __stcg(A.lv[ls].x + mix<D, KR>(t, i), Ls.x[t]);
      __syncthreads();
    }
  }
}

// The V-cycle of the small levels for KR right-hand sides: the cluster levels
// with all of them at once, the one-CTA levels one right-hand side at a time,
// the dense level for all at once.
template <int D, int KR, typename S>
__global__ void __launch_bounds__(TAILM_THREADS) tailm_kernel(const __grid_constant__ TailArgs<float> A,
                                                             float* stash) {
  using V = float;
  constexpr int G = tail_g<D>();
  const int nct = (int)cluster_size(), rank = (int)cluster_rank();
  const int ng = blockDim.x / G;
  const int gg = rank * ng + (int)threadIdx.x / G, NG = nct * ng;
  const int lane = threadIdx.x & (G - 1);
  const int tid = rank * blockDim.x + threadIdx.x, NT = nct * blockDim.x;
  const int l0 = A.l0, ls = A.ls;
  for (int l = l0; l < ls; ++l) {
    const TL<V>& L = A.lv[l];
    tailm_sweep<D, KR, V, S, 0>(L, gg, NG, lane, G);
    for (int base = 0; base < L.nv; base += NG) {
      RowPFM<D, KR, V> st;
      rowm_prefetch<D, KR, V, S, 2>(L, base + gg, base + gg < L.nv, lane, st);
      rowm_finish<D, KR, V, S, 2>(L, base + gg, base + gg < L.nv, lane, G, st);
    }
    cluster_sync_all();
    for (int I = tid; I < L.nvc; I += NT) restrictm_row<D, KR, V>(L, I);
    cluster_sync_all();
  }
  if (A.kd >= 0) {
    tailm_dense_part<D, KR, S>(A, rank, nct, stash);
  } else if (rank == 0) {
    for (int i = 0; i < KR; ++i) tailm_one_cta<D, KR, V, S>(A, i);
  }
  cluster_sync_all();
  for (int l = ls - 1; l >= l0; --l) {
    const TL<V>& L = A.lv[l];
    for (int i = tid; i < L.nv; i += NT) prolongm_row<D, KR, V>(L, i);
    cluster_sync_all();
    tailm_sweep<D, KR, V, S, 1>(L, gg, NG, lane, G);
  }
}

// ------------------------------------------------------------------ outer CG, KR right-hand sides (FP64)

struct CGM {
  CGArgs a;                 // level-0 operator (SELL), permutation, Dirichlet data
  double* U;                // [KR][n] each, solve order
  double* r;
  double* p;
  double* q;
  double* part;             // [KR][pstride] block partials
  double* hist;             // [KR][max_iters]
  Scalars* sc;              // [KR]
  int* ctl;                 // [0]: iteration bodies run
  long long n;
  int pstride;
  unsigned long long cond;  // cudaGraphConditionalHandle (0 = none)
};

// r_i = F_i - A u_D at free dofs, U_i = p_i = 0, res0_i, b_0 of every right-hand side.
template <int D, int KR>
__global__ void __launch_bounds__(CG_THREADS) cgm_init_kernel(CGM m, const double* __restrict__ F, float* b0) {
  const int i = blockIdx.y;
  const long long n = m.n;
  const double* Fi = F + (long long)i * n;
  double* ri = m.r + (long long)i * n;
  double* Ui = m.U + (long long)i * n;
  double* pi = m.p + (long long)i * n;
  double acc = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / D;
    const int c = (int)(t - r * D);
    const long long g = (long long)__ldg(m.a.perm + r) * D + c;
    const double v = __ldg(m.a.isdir + g) ? 0.0 : Fi[g] - __ldg(m.a.lift + g);
    ri[t] = v;
    Ui[t] = 0.0;
    pi[t] = 0.0;
    b0[mix<D, KR>(t, i)] = (float)v;
    acc += v * v;
  }
  if (i == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    m.ctl[0] = 0;
    m.sc[0].abort = 0;
  }
  double tot;
  Scalars* s = m.sc + i;
  if (last_block_sum(acc, m.part + (long long)i * m.pstride, &s->cnt[0], &tot) && threadIdx.x == 0) {
    s->res0 = sqrt(tot);
    s->rr = tot;
    s->relres = 1.0;
    s->iter = 0;
    s->first = 1;
    s->status = 0;
    s->done = (s->res0 == 0.0) ? 1 : 0;
    if (s->done) s->relres = 0.0;
  }
}

// rho_i = r_i . z_i, beta_i (right-hand sides still iterating)
template <int D, int KR>
__global__ void __launch_bounds__(CG_THREADS) cgm_rz_kernel(CGM m, const float* __restrict__ z) {
  const int i = blockIdx.y;
  Scalars* s = m.sc + i;
  if (*(volatile int*)&s->done) return;
  const double* ri = m.r + (long long)i * m.n;
  double acc = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < m.n;
       t += (long long)gridDim.x * blockDim.x)
    acc += ri[t] * (double)__ldcg(z + mix<D, KR>(t, i));
  double tot;
  if (last_block_sum(acc, m.part + (long long)i * m.pstride, &s->cnt[1], &tot) && threadIdx.x == 0) {
    s->beta = s->first ? 0.0 : tot / s->rho;
    s->rho = tot;
    s->first = 0;
  }
}

template <int D, int KR>
__global__ void __launch_bounds__(CG_THREADS) cgm_pupdate_kernel(CGM m, const float* __restrict__ z) {
  const int i = blockIdx.y;
  const Scalars* s = m.sc + i;
  if (s->done) return;
  const double beta = s->beta;
  double* pi = m.p + (long long)i * m.n;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < m.n;
       t += (long long)gridDim.x * blockDim.x)
    pi[t] = (double)__ldcg(z + mix<D, KR>(t, i)) + beta * pi[t];
}

// q_i = A p_i for right-hand sides i0 .. i0+KG-1 (SELL-32, each block read
// once for all of them), p_i . q_i and alpha_i as in spmv_sell_kernel.
template <int D, int KG>
__global__ void __launch_bounds__(CG_THREADS) cgm_spmv_kernel(CGM m, int i0) {
  const CGArgs& a = m.a;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nslices = a.sell_n >> 5;
  double dot[KG];
#pragma unroll
  for (int g = 0; g < KG; ++g) dot[g] = 0.0;
  for (long long s = warp; s < nslices; s += nwarps) {
    const long long base = __ldg(a.sell_ptr + s) + lane;
    const int w = __ldg(a.sell_w + s);
    const int row = __ldg(a.sell_rows + (s << 5) + lane);
    double acc[KG][D];
#pragma unroll
    for (int g = 0; g < KG; ++g)
#pragma unroll
      for (int c = 0; c < D; ++c) acc[g][c] = 0.0;
    for (int k = 0; k < w; ++k) {
      const long long idx = base + ((long long)k << 5);
      const int j = __ldg(a.sell_ci + idx);
      double pj[KG][D];
#pragma unroll
      for (int g = 0; g < KG; ++g)
#pragma unroll
        for (int bb = 0; bb < D; ++bb) pj[g][bb] = m.p[(long long)(i0 + g) * m.n + (long long)j * D + bb];
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int bb = 0; bb < D; ++bb) {
          const double v = __ldg(a.sell_v + (long long)(c * D + bb) * a.sell_tot + idx);
#pragma unroll
          for (int g = 0; g < KG; ++g) acc[g][c] = fma(v, pj[g][bb], acc[g][c]);
        }
    }
    if (row >= 0) {
#pragma unroll
      for (int g = 0; g < KG; ++g)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const long long o = (long long)(i0 + g) * m.n + (long long)row * D + c;
          m.q[o] = acc[g][c];
          dot[g] = fma(acc[g][c], m.p[o], dot[g]);
        }
    }
  }
#pragma unroll
  for (int g = 0; g < KG; ++g) {
    Scalars* s = m.sc + i0 + g;
    double tot;
    if (last_block_sum(dot[g], m.part + (long long)(i0 + g) * m.pstride, &s->cnt[2], &tot) && threadIdx.x == 0 &&
        !s->done) {
      s->pq = tot;
      if (!(tot > 0.0)) {
        s->status = VASMG_ERR_BREAKDOWN;
        s->done = 1;
        s->alpha = 0.0;
      } else {
        s->alpha = s->rho / tot;
      }
    }
  }
}

// U_i += alpha_i p_i, r_i -= alpha_i q_i, ||r_i||, stop test, b_0 of every
// right-hand side still iterating.
template <int D, int KR>
__global__ void __launch_bounds__(CG_THREADS) cgm_update_kernel(CGM m, float* b0) {
  const int i = blockIdx.y;
  Scalars* s = m.sc + i;
  if (*(volatile int*)&s->done) return;
  const double alpha = s->alpha;
  double* Ui = m.U + (long long)i * m.n;
  double* ri = m.r + (long long)i * m.n;
  const double* pi = m.p + (long long)i * m.n;
  const double* qi = m.q + (long long)i * m.n;
  double acc = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < m.n;
       t += (long long)gridDim.x * blockDim.x) {
    Ui[t] += alpha * pi[t];
    const double rv = ri[t] - alpha * qi[t];
    ri[t] = rv;
    b0[mix<D, KR>(t, i)] = (float)rv;
    acc += rv * rv;
  }
  double tot;
  if (last_block_sum(acc, m.part + (long long)i * m.pstride, &s->cnt[3], &tot) && threadIdx.x == 0) {
    s->rr = tot;
    s->relres = sqrt(tot) / s->res0;
    s->iter += 1;
    if (s->iter <= s->max_iters) m.hist[(long long)i * s->max_iters + s->iter - 1] = s->relres;
    if (m.sc[0].abort) {
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
  }
}

// The loop's condition: run another iteration while any right-hand side is
// still iterating.  count: one iteration body has run; more than max_iters + 2
// of them ends every solve with VASMG_ERR_TIMEOUT (a hard bound on the
// device-side loop, independent of the reductions).
template <int KR, bool COND>
__global__ void cgm_cond_kernel(CGM m, int count) {
  if (threadIdx.x != 0) return;
  if (count) m.ctl[0] += 1;
  const bool over = m.ctl[0] > m.sc[0].max_iters + 2;
  int active = 0;
  for (int i = 0; i < KR; ++i) {
    Scalars* s = m.sc + i;
    if (over && !s->done) {
      s->done = 1;
      s->status = VASMG_ERR_TIMEOUT;
    }
    active |= s->done ? 0 : 1;
  }
  if constexpr (COND) {
    if (m.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)m.cond, active ? 1u : 0u);
  }
  m.ctl[1] = active;
}

// U_i (solve order) -> user order with the Dirichlet values written in.
template <int D>
__global__ void cgm_final_kernel(CGM m, double* __restrict__ Uout) {
  const int i = blockIdx.y;
  const double* Ui = m.U + (long long)i * m.n;
  double* Uo = Uout + (long long)i * m.n;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < m.n;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / D;
    const int c = (int)(t - r * D);
    const long long g = (long long)__ldg(m.a.perm + r) * D + c;
    Uo[g] = __ldg(m.a.isdir + g) ? __ldg(m.a.udir + g) : Ui[t];
  }
}

// ------------------------------------------------------------------ engine

template <int D, typename S>
struct MultiEngine : MultiBase {
  using V = float;
  EngineView<V> v;
  int cap = 0;                        // right-hand sides the buffers hold (2, 4 or 8)
  std::vector<DevBuf<V>> xm, bm, rm;  // per level, [nv][cap][D] (a pass with KR uses the first nv KR D)
  DevBuf<double> U, r, p, q, Fb, Ub, part, hist;
  DevBuf<Scalars> sc;
  DevBuf<int> ctl;
  DevBuf<V> stash;
  Scalars* host_sc = nullptr;
  int* host_ctl = nullptr;
  int pstride = 1;
  cudaGraphExec_t exec_while[4] = {nullptr, nullptr, nullptr, nullptr};  // by log2(KR)
  cudaGraphExec_t exec_body[4] = {nullptr, nullptr, nullptr, nullptr};
  i64 launches_body[4] = {0, 0, 0, 0};
  i64 launch_counter = 0;
  unsigned long long cond = 0;

  explicit MultiEngine(const EngineView<V>& view) : v(view) {}
  ~MultiEngine() override {
    for (int t = 0; t < 4; ++t) {
      if (exec_while[t]) cudaGraphExecDestroy(exec_while[t]);
      if (exec_body[t]) cudaGraphExecDestroy(exec_body[t]);
    }
    if (host_sc) cudaFreeHost(host_sc);
    if (host_ctl) cudaFreeHost(host_ctl);
  }
  void set_view(const EngineView<V>& view) override { v = view; }

  static int slot(int KR) { return KR == 2 ? 1 : (KR == 4 ? 2 : 3); }
  i64 n0() const { return v.nv[0] * D; }

  // Buffers for passes of up to kr right-hand sides; growing them drops the
  // graphs captured with the old ones.
  void allocate(int kr) {
    if (kr <= cap) return;
    for (int t = 0; t < 4; ++t) {
      if (exec_while[t]) cudaGraphExecDestroy(exec_while[t]);
      if (exec_body[t]) cudaGraphExecDestroy(exec_body[t]);
      exec_while[t] = exec_body[t] = nullptr;
    }
    cudaStream_t s = v.stream;
    VASMG_CUDA(cudaStreamSynchronize(s));
    xm.resize(v.L);
    bm.resize(v.L);
    rm.resize(v.L);
    for (int l = 0; l < v.L; ++l) {
      const i64 n = std::max<i64>(1, v.nv[l] * D * kr);
      xm[l].alloc(n, s);
      bm[l].alloc(n, s);
      rm[l].alloc(n, s);
      xm[l].zero();
      bm[l].zero();
      rm[l].zero();
    }
    const i64 n = n0();
    U.alloc(n * kr, s);
    r.alloc(n * kr, s);
    p.alloc(n * kr, s);
    q.alloc(n * kr, s);
    Fb.alloc(n * kr, s);
    Ub.alloc(n * kr, s);
    p.zero();
    pstride = std::max(v.cg_blocks, v.spmv_blocks);
    part.alloc((i64)pstride * kr, s);
    hist.alloc((i64)std::max(1, v.max_iters) * kr, s);
    sc.alloc(kr, s);
    sc.zero();
    ctl.alloc(2, s);
    ctl.zero();
    // the one-CTA levels above the dense level, saved per right-hand side
    const TailArgs<V>& ta = v.ta;
    i64 slen = 1;
    if (ta.kd > ta.ls) slen = ta.soff[ta.kd] - ta.soff[ta.ls];
    stash.alloc(std::max<i64>(1, slen) * kr, s);
    if (!host_sc) VASMG_CUDA(cudaMallocHost((void**)&host_sc, sizeof(Scalars) * KMAX));
    if (!host_ctl) VASMG_CUDA(cudaMallocHost((void**)&host_ctl, sizeof(int) * 2));
    cap = kr;
  }

  // level l's view with the multi vectors of KR right-hand sides
  LV<V> lvm(int l) const {
    LV<V> a = v.lv[l];
    a.x = xm[l].get();
    a.b = bm[l].get();
    a.r = rm[l].get();
    if (l + 1 < v.L) {
      a.bc = bm[l + 1].get();
      a.xc = xm[l + 1].get();
    }
    return a;
  }
  CGM cgm() const {
    CGM m;
    m.a = v.cga;
    m.U = U.get();
    m.r = r.get();
    m.p = p.get();
    m.q = q.get();
    m.part = part.get();
    m.hist = hist.get();
    m.sc = sc.get();
    m.ctl = ctl.get();
    m.n = n0();
    m.pstride = pstride;
    m.cond = cond;
    return m;
  }

  int plain_grid(i64 threads) const { return (int)std::max<i64>(1, std::min<i64>(ceil_div(threads, 256), v.sms * 8)); }

  template <typename K>
  void coop(K kern, int grid, const LV<V>& a, int G, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(dfm_threads<D, V>());
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    Scalars* scp = sc.get();
    VASMG_CUDA(cudaLaunchKernelEx(&cfg, kern, a, scp, G));
    ++launch_counter;
  }

  // The staged sweeps with KR right-hand sides (3D): whether their grids of
  // R CTAs fit the device (measured once per KR; the shared-memory limit is
  // raised first).
  int stg_cap[4] = {-1, -1, -1, -1};
  template <int KR>
  bool staged_fits(int R) {
    if constexpr (D == 3) {
      int& cap_kr = stg_cap[slot(KR)];
      if (cap_kr < 0) {
        const int smem = stg_smem_bytes<S>();
        VASMG_CUDA(cudaFuncSetAttribute(vstagedm_kernel<D, KR, V, S, 0>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        VASMG_CUDA(cudaFuncSetAttribute(vstagedm_kernel<D, KR, V, S, 1>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int bd = 0, bu = 0;
        VASMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bd, vstagedm_kernel<D, KR, V, S, 0>, STG_T + 32,
                                                                 smem));
        VASMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu, vstagedm_kernel<D, KR, V, S, 1>, STG_T + 32,
                                                                 smem));
        cap_kr = std::min(bd, bu) * v.sms;
      }
      return cap_kr >= R;
    } else {
      (void)R;
      return false;
    }
  }
  template <typename K>
  void coop_staged(K kern, int grid, const LV<V>& a, const void* op, int G, cudaStream_t s) {
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
    const StagedOp<S> o = *static_cast<const StagedOp<S>*>(op);
    VASMG_CUDA(cudaLaunchKernelEx(&cfg, kern, a, o, scp, G));
    ++launch_counter;
  }
  // level l's sweep in direction MODE from the staged copy, if it has one that fits
  template <int KR, int MODE>
  bool sweep_staged(int l, const LV<V>& a, cudaStream_t s) {
    if constexpr (D == 3) {
      const std::vector<const void*>& ops = MODE == 0 ? v.stg_fwd : v.stg_bwd;
      if (l >= (int)ops.size() || !ops[l] || !staged_fits<KR>(a.R)) return false;
      coop_staged(vstagedm_kernel<D, KR, V, S, MODE>, a.R, a, ops[l], v.G[l], s);
      return true;
    } else {
      (void)l;
      (void)a;
      (void)s;
      return false;
    }
  }

  // phases: 1 forward sweep, 2 residual, 4 restriction
  template <int KR>
  void down(int l, int phases, cudaStream_t s) {
    const LV<V> a = lvm(l);
    if ((phases & 1) && !sweep_staged<KR, 0>(l, a, s)) coop(vdownm_kernel<D, KR, V, S>, a.R, a, v.G[l], s);
    if (phases & 2) {
      residualm_kernel<D, KR, V, S><<<plain_grid((i64)a.nv * v.G[l]), 256, 0, s>>>(a, v.G[l]);
      ++launch_counter;
    }
    if (phases & 4) {
      restrictm_kernel<D, KR, V><<<plain_grid(a.nvc), 256, 0, s>>>(a);
      ++launch_counter;
    }
  }
  // phases: 1 prolongation, 2 backward sweep
  template <int KR>
  void up(int l, int phases, cudaStream_t s) {
    const LV<V> a = lvm(l);
    if (phases & 1) {
      prolongm_kernel<D, KR, V><<<plain_grid(a.nv), 256, 0, s>>>(a);
      ++launch_counter;
    }
    if ((phases & 2) && !sweep_staged<KR, 1>(l, a, s)) coop(vupm_kernel<D, KR, V, S>, a.R, a, v.G[l], s);
  }
  template <int KR>
  size_t tail_smem_bytes() const {
    size_t smem = v.tail_smem;
    if (v.ta.kd >= 0 && v.ta.kd >= v.ta.ls) smem = (size_t)v.ta.dsoff * sizeof(V) + sizeof(V) * (size_t)KR * v.ta.dld;
    return smem;
  }
  template <int KR>
  void tail(cudaStream_t s) {
    TailArgs<V> ta = v.ta;
    for (int l = 0; l < v.L; ++l) {
      ta.lv[l].x = xm[l].get();
      ta.lv[l].b = bm[l].get();
      ta.lv[l].r = rm[l].get();
      if (l + 1 < v.L) {
        ta.lv[l].bc = bm[l + 1].get();
        ta.lv[l].xc = xm[l + 1].get();
      }
    }
    const size_t smem = tail_smem_bytes<KR>();
    VASMG_CHECK(smem <= (size_t)TAIL_SMEM_MAX, VASMG_ERR_UNSUPPORTED,
                "tail levels too large for shared memory with this many right-hand sides");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(v.nct);
    cfg.blockDim = dim3(TAILM_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = v.nct;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    VASMG_CUDA(cudaLaunchKernelEx(&cfg, tailm_kernel<D, KR, S>, ta, stash.get()));
    ++launch_counter;
  }
  template <int KR>
  void vcycle(cudaStream_t s) {
    for (int l = 0; l < v.lt; ++l) down<KR>(l, 7, s);
    tail<KR>(s);
    for (int l = v.lt - 1; l >= 0; --l) up<KR>(l, 3, s);
  }
  template <int KR, bool COND>
  void body(cudaStream_t s) {
    const CGM m = cgm();
    V* z = xm[0].get();
    const dim3 g(v.cg_blocks, KR);
    vcycle<KR>(s);
    cgm_rz_kernel<D, KR><<<g, CG_THREADS, 0, s>>>(m, z);
    cgm_pupdate_kernel<D, KR><<<g, CG_THREADS, 0, s>>>(m, z);
    for (int i0 = 0; i0 < KR; i0 += KG_SPMV) {
      if (KR - i0 >= KG_SPMV) {
        cgm_spmv_kernel<D, KG_SPMV><<<v.spmv_blocks, CG_THREADS, 0, s>>>(m, i0);
      } else {
        cgm_spmv_kernel<D, 2><<<v.spmv_blocks, CG_THREADS, 0, s>>>(m, i0);
      }
      ++launch_counter;
    }
    cgm_update_kernel<D, KR><<<g, CG_THREADS, 0, s>>>(m, bm[0].get());
    cgm_cond_kernel<KR, COND><<<1, 32, 0, s>>>(m, 1);
    launch_counter += 4;
  }

  template <int KR>
  void set_attributes() {
    VASMG_CUDA(cudaFuncSetAttribute(tailm_kernel<D, KR, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, TAIL_SMEM_MAX));
    if (v.nct > 8)
      VASMG_CUDA(cudaFuncSetAttribute(tailm_kernel<D, KR, S>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    // every region of a level must be resident at once: the multi sweep CTAs
    // must fit as many per SM as the single sweeps' regions need
    int bd = 0, bu = 0;
    VASMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bd, vdownm_kernel<D, KR, V, S>, dfm_threads<D, V>(), 0));
    VASMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu, vupm_kernel<D, KR, V, S>, dfm_threads<D, V>(), 0));
    for (int l = 0; l < v.lt; ++l)
      VASMG_CHECK((i64)std::min(bd, bu) * v.sms >= v.lv[l].R, VASMG_ERR_UNSUPPORTED,
                  "the multi-right-hand-side sweep cannot hold the level's regions");
  }

  template <int KR>
  bool build_while(int t) {
    cudaStream_t s = v.stream;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
    bool ok = true;
    cudaGraphConditionalHandle h = 0;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) ok = false;
    cudaGraph_t out = nullptr;
    cudaGraphNode_t init_node = nullptr, wnode = nullptr;
    if (ok) {
      cond = (unsigned long long)h;
      ok = cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const CGM m = cgm();
        cgm_init_kernel<D, KR><<<dim3(v.cg_blocks, KR), CG_THREADS, 0, s>>>(m, Fb.get(), bm[0].get());
        cgm_cond_kernel<KR, true><<<1, 32, 0, s>>>(m, 0);
        ok = cudaStreamEndCapture(s, &out) == cudaSuccess;
      }
    }
    if (ok) {
      size_t nn = 0;
      ok = cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn == 2;
      if (ok) {
        cudaGraphNode_t nodes[2];
        ok = cudaGraphGetNodes(g, nodes, &nn) == cudaSuccess;
        // the WHILE node follows the condition kernel (which follows init)
        if (ok) {
          cudaKernelNodeParams kp = {};
          ok = cudaGraphKernelNodeGetParams(nodes[1], &kp) == cudaSuccess;
          init_node = (ok && kp.func == (void*)cgm_cond_kernel<KR, true>) ? nodes[1] : nodes[0];
        }
      }
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
            body<KR, true>(s);
          } catch (...) {
            ok = false;
          }
          ok = (cudaStreamEndCapture(s, &out) == cudaSuccess) && ok;
        }
        launches_body[t] = launch_counter;
      }
    }
    if (ok) {
      ok = cudaStreamBeginCaptureToGraph(s, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        cgm_final_kernel<D><<<dim3(v.cg_blocks, KR), CG_THREADS, 0, s>>>(cgm(), Ub.get());
        ok = cudaStreamEndCapture(s, &out) == cudaSuccess;
      }
    }
    if (ok && cudaGraphInstantiate(&exec_while[t], g, 0) != cudaSuccess) {
      exec_while[t] = nullptr;
      ok = false;
    }
    cudaGraphDestroy(g);
    cudaGetLastError();
    cond = 0;
    return ok;
  }

  template <int KR>
  void build_body(int t) {
    cudaStream_t s = v.stream;
    cudaGraph_t bg = nullptr;
    launch_counter = 0;
    cond = 0;
    VASMG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
      body<KR, false>(s);
    } catch (...) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(s, &junk);
      if (junk) cudaGraphDestroy(junk);
      cudaGetLastError();
      throw;
    }
    VASMG_CUDA(cudaStreamEndCapture(s, &bg));
    launches_body[t] = launch_counter;
    VASMG_CUDA(cudaGraphInstantiate(&exec_body[t], bg, 0));
    cudaGraphDestroy(bg);
  }

  // One pass: KR right-hand sides (kc of them real, the rest zero).
  template <int KR>
  int pass(int kc, const double* const* F, double* const* Uo, double tol, vasmg_stats* st, i64* launches) {
    cudaStream_t s = v.stream;
    const int t = slot(KR);
    if (!exec_while[t] && !exec_body[t]) {
      set_attributes<KR>();
      if (!(v.use_graph && build_while<KR>(t))) build_body<KR>(t);
    }
    const i64 n = n0();
    std::vector<Scalars> init(KR);
    for (int i = 0; i < KR; ++i) {
      std::memset(&init[i], 0, sizeof(Scalars));
      init[i].tol = tol;
      init[i].max_iters = v.max_iters;
    }
    VASMG_CUDA(cudaMemcpyAsync(sc.get(), init.data(), sizeof(Scalars) * KR, cudaMemcpyHostToDevice, s));
    for (int i = 0; i < KR; ++i) {
      if (i < kc)
        VASMG_CUDA(cudaMemcpyAsync(Fb.get() + (i64)i * n, F[i], sizeof(double) * n, cudaMemcpyDefault, s));
      else
        VASMG_CUDA(cudaMemsetAsync(Fb.get() + (i64)i * n, 0, sizeof(double) * n, s));
    }
    i64 bodies = 0;
    if (exec_while[t]) {
      VASMG_CUDA(cudaGraphLaunch(exec_while[t], s));
    } else {
      const CGM m = cgm();
      cgm_init_kernel<D, KR><<<dim3(v.cg_blocks, KR), CG_THREADS, 0, s>>>(m, Fb.get(), bm[0].get());
      cgm_cond_kernel<KR, false><<<1, 32, 0, s>>>(m, 0);
      check_launch("cgm_init");
      VASMG_CUDA(cudaMemcpyAsync(host_ctl, ctl.get(), sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
      VASMG_CUDA(cudaStreamSynchronize(s));
      while (host_ctl[1] && bodies <= v.max_iters + 2) {
        VASMG_CUDA(cudaGraphLaunch(exec_body[t], s));
        VASMG_CUDA(cudaMemcpyAsync(host_ctl, ctl.get(), sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
        VASMG_CUDA(cudaStreamSynchronize(s));
        ++bodies;
      }
      cgm_final_kernel<D><<<dim3(v.cg_blocks, KR), CG_THREADS, 0, s>>>(m, Ub.get());
      check_launch("cgm_final");
    }
    VASMG_CUDA(cudaMemcpyAsync(host_sc, sc.get(), sizeof(Scalars) * KR, cudaMemcpyDeviceToHost, s));
    VASMG_CUDA(cudaMemcpyAsync(host_ctl, ctl.get(), sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    for (int i = 0; i < kc; ++i)
      VASMG_CUDA(cudaMemcpyAsync(Uo[i], Ub.get() + (i64)i * n, sizeof(double) * n, cudaMemcpyDefault, s));
    VASMG_CUDA(cudaStreamSynchronize(s));
    if (launches) *launches += 2 + 2 + launches_body[t] * (i64)host_ctl[0];
    int worst = VASMG_OK;
    for (int i = 0; i < kc; ++i) {
      const Scalars& h = host_sc[i];
      int rc = h.status;
      if (host_sc[0].abort) rc = VASMG_ERR_TIMEOUT;
      if (st) {
        st[i].iterations = h.iter;
        st[i].rel_res = h.relres;
        st[i].n_levels = v.L;
        if (st[i].res_history && st[i].res_history_cap > 0) {
          const int kk = std::min(st[i].res_history_cap, std::min(h.iter, v.max_iters));
          if (kk > 0)
            VASMG_CUDA(cudaMemcpy(st[i].res_history, hist.get() + (i64)i * v.max_iters, sizeof(double) * kk,
                                  cudaMemcpyDeviceToHost));
        }
      }
      if (rc < 0) worst = std::min(worst, rc);  // errors first
      else if (worst >= 0) worst = std::max(worst, rc);
    }
    return worst;
  }

  int solve(int k, const double* const* F, double* const* Uo, double tol, vasmg_stats* st, i64* launches) override {
    allocate(k <= 2 ? 2 : (k <= 4 ? 4 : KMAX));
    int worst = VASMG_OK;
    for (int c0 = 0; c0 < k; c0 += KMAX) {
      const int kc = std::min(KMAX, k - c0);
      vasmg_stats* sti = st ? st + c0 : nullptr;
      int rc;
      if (kc <= 2) rc = pass<2>(kc, F + c0, Uo + c0, tol, sti, launches);
      else if (kc <= 4) rc = pass<4>(kc, F + c0, Uo + c0, tol, sti, launches);
      else rc = pass<8>(kc, F + c0, Uo + c0, tol, sti, launches);
      if (rc < 0) worst = std::min(worst, rc);
      else if (worst >= 0) worst = std::max(worst, rc);
    }
    return worst;
  }

  // ---------------------------------------------------------------- timing
  // Algorithmic bytes of one launch with KR right-hand sides: the operator
  // arrays once, every vector entry once per right-hand side.
  double blocks_bytes(i64 nblocks) const { return (double)nblocks * (D * D * sizeof(S) + 4.0); }
  template <int KR>
  double bytes_of(int which, int l) const {
    const LV<V>& a = v.lv[l];
    const double nv = (double)a.nv, n = nv * D, nlo = (double)a.nlo, nnz = (double)a.nnz;
    const double vec = sizeof(V) * (double)KR;
    switch (which) {
      case VASMG_KERNEL_FWD_SWEEP: return blocks_bytes((i64)nlo) + 8.0 * nv + nv * D * D * sizeof(V) + 3.0 * n * vec;
      case VASMG_KERNEL_SWEEP: return blocks_bytes((i64)nnz) + 8.0 * nv + 4.0 + nv * D * D * sizeof(V) + 3.0 * n * vec;
      case VASMG_KERNEL_RESIDUAL: return blocks_bytes((i64)(nnz - nlo)) + 8.0 * nv + 2.0 * n * vec;
      case VASMG_KERNEL_RESTRICT:
        return v.pnnz[l] * (4.0 + sizeof(V)) + (v.nv[l + 1] + 1.0) * 4.0 + n * vec + (double)v.nv[l + 1] * D * vec;
      case VASMG_KERNEL_PROLONG:
        return v.pnnz[l] * (4.0 + sizeof(V)) + (nv + 1.0) * 4.0 + nv + (double)v.nv[l + 1] * D * vec + 2.0 * n * vec;
      case VASMG_KERNEL_SPMV64:
        return (double)v.sell_real_entries * (D * D * 8.0 + 4.0) + 3.0 * 8.0 * (double)n0() * KR;
      default: return 0.0;
    }
  }
  template <int KR>
  double time_k(int which, int level, int reps, double* bytes) {
    cudaStream_t s = v.stream;
    VASMG_CHECK(which == VASMG_KERNEL_SPMV64 || which == VASMG_KERNEL_VCYCLE || which == VASMG_KERNEL_TAIL ||
                    (level < v.lt && level + 1 < v.L),
                VASMG_ERR_INVALID_ARG, "not a region level");
    set_attributes<KR>();
    VASMG_CUDA(cudaMemsetAsync(&sc.get()->abort, 0, sizeof(int), s));
    const CGM m = cgm();
    auto run = [&]() {
      switch (which) {
        case VASMG_KERNEL_FWD_SWEEP: down<KR>(level, 1, s); break;
        case VASMG_KERNEL_RESIDUAL: down<KR>(level, 2, s); break;
        case VASMG_KERNEL_RESTRICT: down<KR>(level, 4, s); break;
        case VASMG_KERNEL_PROLONG: up<KR>(level, 1, s); break;
        case VASMG_KERNEL_SWEEP: up<KR>(level, 2, s); break;
        case VASMG_KERNEL_TAIL: tail<KR>(s); break;
        case VASMG_KERNEL_VCYCLE: vcycle<KR>(s); break;
        case VASMG_KERNEL_SPMV64:
          for (int i0 = 0; i0 < KR; i0 += KG_SPMV) {
            if (KR - i0 >= KG_SPMV) cgm_spmv_kernel<D, KG_SPMV><<<v.spmv_blocks, CG_THREADS, 0, s>>>(m, i0);
            else cgm_spmv_kernel<D, 2><<<v.spmv_blocks, CG_THREADS, 0, s>>>(m, i0);
          }
          break;
        default: throw Error(VASMG_ERR_INVALID_ARG, "unknown kernel");
      }
    };
    run();
    check_launch("multi timing");
    VASMG_CUDA(cudaStreamSynchronize(s));
    cudaEvent_t e0, e1;
    VASMG_CUDA(cudaEventCreate(&e0));
    VASMG_CUDA(cudaEventCreate(&e1));
    VASMG_CUDA(cudaEventRecord(e0, s));
    for (int i = 0; i < reps; ++i) run();
    VASMG_CUDA(cudaEventRecord(e1, s));
    VASMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    VASMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int ab = 0;
    VASMG_CUDA(cudaMemcpy(&ab, &sc.get()->abort, sizeof(int), cudaMemcpyDeviceToHost));
    VASMG_CHECK(ab == 0, VASMG_ERR_TIMEOUT, "a device wait gave up");
    double b = 0.0;
    if (which == VASMG_KERNEL_VCYCLE) {
      for (int l = 0; l < v.lt; ++l)
        b += bytes_of<KR>(VASMG_KERNEL_FWD_SWEEP, l) + bytes_of<KR>(VASMG_KERNEL_RESIDUAL, l) +
             bytes_of<KR>(VASMG_KERNEL_RESTRICT, l) + bytes_of<KR>(VASMG_KERNEL_PROLONG, l) +
             bytes_of<KR>(VASMG_KERNEL_SWEEP, l);
    } else if (which != VASMG_KERNEL_TAIL) {
      b = bytes_of<KR>(which, level);
    }
    *bytes = b;
    return (double)ms / reps;
  }
  double time(int which, int level, int k, int reps, double* bytes) override {
    allocate(k);
    switch (k) {
      case 2: return time_k<2>(which, level, reps, bytes);
      case 4: return time_k<4>(which, level, reps, bytes);
      case 8: return time_k<8>(which, level, reps, bytes);
      default: throw Error(VASMG_ERR_INVALID_ARG, "k must be 2, 4 or 8");
    }
  }
};

// ------------------------------------------------------------------ several hierarchies per launch

// One hierarchy's region level in a batched launch: its CTAs are
// [cta0, cta0 + nb) of the grid (nb = its regions for the sweeps, its blocks
// for the plain kernels).
struct BatchItem {
  LV<float> lv;
  int dim, G, cta0, nb;
};

__device__ __forceinline__ int batch_item_of(const BatchItem* __restrict__ it, int n, int b) {
  int i = 0;
  while (i + 1 < n && it[i + 1].cta0 <= b) ++i;
  return i;
}

// Region k's forward sweep from zero (MODE 0) or backward sweep (MODE 1):
// the steps of vdownm_kernel / vupm_kernel with one right-hand side, the exit
// counted over this hierarchy's R regions.
template <int D, typename S, int MODE>
__device__ __forceinline__ void sweep_region(const LV<float>& L, int k, int G, int R, int* abort_flag) {
  using V = float;
  __shared__ unsigned s_epoch;
  if (threadIdx.x == 0) s_epoch = *(volatile unsigned*)(L.ctr + (MODE == 0 ? C_DEPOCH : C_UEPOCH));
  __syncthreads();
  const unsigned epoch = s_epoch;
  const int C = L.ncol;
  const int g = threadIdx.x / G, lane = threadIdx.x & (G - 1);
  const int nb0 = __ldg(L.nb_rp + k), nnb = __ldg(L.nb_rp + k + 1) - nb0;
  unsigned long long* pg = MODE == 0 ? L.pg_d : L.pg_u;
  unsigned long long* mine = pg + k;
  unsigned stage = 0;
  for (int i = 0; i < C; ++i) {
    const int c = MODE == 0 ? i : C - 1 - i;
    const int r0 = __ldg(L.RS + c * (R + 1) + k), r1 = __ldg(L.RS + c * (R + 1) + k + 1);
    if (r0 < r1) {
      RowPFM<D, 1, V> cur;
      rowm_prefetch<D, 1, V, S, MODE>(L, r0 + g, r0 + g < r1, lane, cur);
      if (stage > 0 && !wait_regions(L.nb + nb0, nnb, pg, epoch, stage, abort_flag)) break;
      rowsm_pipelined<D, 1, V, S, MODE>(L, r0, r1, G, cur);
    }
    publish_stage(mine, epoch, ++stage);
  }
  leave(L.ctr, MODE == 0 ? C_DEXIT : C_UEXIT, MODE == 0 ? C_DEPOCH : C_UEPOCH, R);
}

template <typename S, int MODE>
__global__ void __launch_bounds__(DFM_THREADS, 2) sweepb_kernel(const BatchItem* __restrict__ items, int nitems,
                                                               int* abort_flag) {
  const BatchItem& it = items[batch_item_of(items, nitems, blockIdx.x)];
  if (it.dim == 2) sweep_region<2, S, MODE>(it.lv, blockIdx.x - it.cta0, it.G, it.nb, abort_flag);
  else sweep_region<3, S, MODE>(it.lv, blockIdx.x - it.cta0, it.G, it.nb, abort_flag);
}

template <int D, typename S>
__device__ __forceinline__ void residual_rows(const LV<float>& L, int lb, int nb, int G) {
  const int NG = DFM_THREADS / G;
  const int g = threadIdx.x / G, lane = threadIdx.x & (G - 1);
  for (int base = lb * NG; base < L.nv; base += nb * NG) {
    RowPFM<D, 1, float> st;
    rowm_prefetch<D, 1, float, S, 2>(L, base + g, base + g < L.nv, lane, st);
    rowm_finish<D, 1, float, S, 2>(L, base + g, base + g < L.nv, lane, G, st);
  }
}

template <typename S>
__global__ void __launch_bounds__(DFM_THREADS) residualb_kernel(const BatchItem* __restrict__ items, int nitems) {
  const BatchItem& it = items[batch_item_of(items, nitems, blockIdx.x)];
  const int lb = blockIdx.x - it.cta0;
  if (it.dim == 2) residual_rows<2, S>(it.lv, lb, it.nb, it.G);
  else residual_rows<3, S>(it.lv, lb, it.nb, it.G);
}

// PHASE 0: b_{l+1} = R r_l, 1: x_l += P x_{l+1}, thread per row
template <int PHASE>
__global__ void __launch_bounds__(DFM_THREADS) transferb_kernel(const BatchItem* __restrict__ items, int nitems) {
  const BatchItem& it = items[batch_item_of(items, nitems, blockIdx.x)];
  const LV<float>& L = it.lv;
  const int lb = blockIdx.x - it.cta0, stride = it.nb * blockDim.x;
  const int n = PHASE == 0 ? L.nvc : L.nv;
  for (int i = lb * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (PHASE == 0) {
      if (it.dim == 2) restrictm_row<2, 1, float>(L, i);
      else restrictm_row<3, 1, float>(L, i);
    } else {
      if (it.dim == 2) prolongm_row<2, 1, float>(L, i);
      else prolongm_row<3, 1, float>(L, i);
    }
  }
}

// Every hierarchy's tail: cluster c runs hierarchy c's levels from its own
// first tail level down and back.
template <typename S>
__global__ void __launch_bounds__(TAIL_THREADS) tailb_kernel(const TailArgs<float>* __restrict__ args,
                                                             const int* __restrict__ dims) {
  const int c = blockIdx.x / (int)cluster_size();
  if (dims[c] == 2) tail_run<2, float, S>(args[c]);
  else tail_run<3, float, S>(args[c]);
}

// One hierarchy's outer CG in a batched launch (its own vectors, scalars and
// partials; its own grid sizes, so its reductions are those of vasmg_solve).
struct CGB {
  CGArgs a;
  float* b0;          // level-0 b of its V-cycle
  const float* z;     // level-0 x of its V-cycle
  const double* F;    // user order
  double* Uout;       // user order
  int dim, cg_blocks, spmv_blocks;
};

__global__ void __launch_bounds__(CG_THREADS) cgb_init_kernel(const CGB* __restrict__ items) {
  const CGB& m = items[blockIdx.y];
  if ((int)blockIdx.x >= m.cg_blocks) return;
  const CGArgs& a = m.a;
  const int D = m.dim;
  const long long n = (long long)a.nv * D;
  double acc = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)m.cg_blocks * blockDim.x) {
    const long long r = t / D;
    const int c = (int)(t - r * D);
    const long long g = (long long)__ldg(a.perm + r) * D + c;
    const double v = __ldg(a.isdir + g) ? 0.0 : m.F[g] - __ldg(a.lift + g);
    a.r[t] = v;
    a.U[t] = 0.0;
    a.p[t] = 0.0;
    m.b0[t] = (float)v;
    acc += v * v;
  }
  double tot;
  if (last_block_sum(acc, a.part, &a.sc->cnt[0], &tot, m.cg_blocks, blockIdx.x) && threadIdx.x == 0) {
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
  }
}

__global__ void __launch_bounds__(CG_THREADS) cgb_rz_kernel(const CGB* __restrict__ items) {
  const CGB& m = items[blockIdx.y];
  if ((int)blockIdx.x >= m.cg_blocks) return;
  const CGArgs& a = m.a;
  Scalars* s = a.sc;
  if (*(volatile int*)&s->done) return;
  const long long n = (long long)a.nv * m.dim;
  double acc = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)m.cg_blocks * blockDim.x)
    acc += a.r[t] * (double)__ldcg(m.z + t);
  double tot;
  if (last_block_sum(acc, a.part, &s->cnt[1], &tot, m.cg_blocks, blockIdx.x) && threadIdx.x == 0) {
    s->beta = s->first ? 0.0 : tot / s->rho;
    s->rho = tot;
    s->first = 0;
  }
}

__global__ void __launch_bounds__(CG_THREADS) cgb_pupdate_kernel(const CGB* __restrict__ items) {
  const CGB& m = items[blockIdx.y];
  if ((int)blockIdx.x >= m.cg_blocks) return;
  const CGArgs& a = m.a;
  if (a.sc->done) return;
  const double beta = a.sc->beta;
  const long long n = (long long)a.nv * m.dim;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)m.cg_blocks * blockDim.x)
    a.p[t] = (double)__ldcg(m.z + t) + beta * a.p[t];
}

template <int D>
__device__ __forceinline__ void spmv_rows(const CGB& m) {
  const CGArgs& a = m.a;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)m.spmv_blocks * blockDim.x) >> 5;
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
  double tot;
  if (last_block_sum(dot, a.part, &a.sc->cnt[2], &tot, m.spmv_blocks, blockIdx.x) && threadIdx.x == 0) {
    Scalars* s = a.sc;
    if (!s->done) {
      s->pq = tot;
      if (!(tot > 0.0)) {
        s->status = VASMG_ERR_BREAKDOWN;
        s->done = 1;
        s->alpha = 0.0;
      } else {
        s->alpha = s->rho / tot;
      }
    }
  }
}

__global__ void __launch_bounds__(CG_THREADS) cgb_spmv_kernel(const CGB* __restrict__ items) {
  const CGB& m = items[blockIdx.y];
  if ((int)blockIdx.x >= m.spmv_blocks) return;
  if (m.dim == 2) spmv_rows<2>(m);
  else spmv_rows<3>(m);
}

__global__ void __launch_bounds__(CG_THREADS) cgb_update_kernel(const CGB* __restrict__ items,
                                                                const int* __restrict__ abort_flag) {
  const CGB& m = items[blockIdx.y];
  if ((int)blockIdx.x >= m.cg_blocks) return;
  const CGArgs& a = m.a;
  Scalars* s = a.sc;
  if (*(volatile int*)&s->done) return;
  const double alpha = s->alpha;
  const long long n = (long long)a.nv * m.dim;
  double acc = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)m.cg_blocks * blockDim.x) {
    a.U[t] += alpha * a.p[t];
    const double rv = a.r[t] - alpha * a.q[t];
    a.r[t] = rv;
    m.b0[t] = (float)rv;
    acc += rv * rv;
  }
  double tot;
  if (last_block_sum(acc, a.part, &s->cnt[3], &tot, m.cg_blocks, blockIdx.x) && threadIdx.x == 0) {
    s->rr = tot;
    s->relres = sqrt(tot) / s->res0;
    s->iter += 1;
    if (s->iter <= s->max_iters) a.hist[s->iter - 1] = s->relres;
    if (*(volatile const int*)abort_flag) {
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
  }
}

// Another iteration while any hierarchy is still iterating; more than
// max_iters + 2 bodies end every solve with VASMG_ERR_TIMEOUT.  ctl[0]:
// bodies run, ctl[1]: any active.
template <bool COND>
__global__ void cgb_cond_kernel(const CGB* __restrict__ items, int nitems, int* ctl, int max_iters,
                                unsigned long long cond, int count) {
  if (threadIdx.x != 0) return;
  if (count) ctl[0] += 1;
  const bool over = ctl[0] > max_iters + 2;
  int active = 0;
  for (int i = 0; i < nitems; ++i) {
    Scalars* s = items[i].a.sc;
    if (over && !s->done) {
      s->done = 1;
      s->status = VASMG_ERR_TIMEOUT;
    }
    active |= s->done ? 0 : 1;
  }
  if constexpr (COND) {
    if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, active ? 1u : 0u);
  }
  ctl[1] = active;
}

__global__ void __launch_bounds__(CG_THREADS) cgb_final_kernel(const CGB* __restrict__ items) {
  const CGB& m = items[blockIdx.y];
  if ((int)blockIdx.x >= m.cg_blocks) return;
  const CGArgs& a = m.a;
  const int D = m.dim;
  const long long n = (long long)a.nv * D;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)m.cg_blocks * blockDim.x) {
    const long long r = t / D;
    const int c = (int)(t - r * D);
    const long long g = (long long)__ldg(a.perm + r) * D + c;
    m.Uout[g] = __ldg(a.isdir + g) ? __ldg(a.udir + g) : a.U[t];
  }
}

template <typename S>
int batch_sweep_capacity() {
  int dev = 0, sms = 0, bd = 0, bu = 0;
  VASMG_CUDA(cudaGetDevice(&dev));
  VASMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  VASMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bd, sweepb_kernel<S, 0>, DFM_THREADS, 0));
  VASMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu, sweepb_kernel<S, 1>, DFM_THREADS, 0));
  return std::min(bd, bu) * sms;
}

template <typename S>
struct BatchRun {
  const std::vector<EngineView<float>>& v;
  cudaStream_t s;
  int n = 0, maxlt = 0, nct = 1, sms = 1, max_iters = 1;
  size_t tail_smem = 0;
  // device tables
  std::vector<DevBuf<BatchItem>> sweep_items, plain_items, restrict_items, prolong_items;
  std::vector<int> sweep_items_n, sweep_ctas, plain_ctas, restrict_ctas, prolong_ctas;
  DevBuf<TailArgs<float>> targs;
  DevBuf<int> tdims, ctl, abort_flag;
  DevBuf<CGB> cg;
  int cg_grid = 1, spmv_grid = 1;
  i64 launches = 0;
  unsigned long long cond = 0;

  BatchRun(const std::vector<EngineView<float>>& views, cudaStream_t stream) : v(views), s(stream) {
    n = (int)v.size();
    int dev = 0;
    VASMG_CUDA(cudaGetDevice(&dev));
    VASMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (const auto& e : v) {
      maxlt = std::max(maxlt, e.lt);
      nct = std::max(nct, e.nct);
      max_iters = std::max(max_iters, e.max_iters);
      size_t sm = e.tail_smem;
      if (e.ta.kd >= 0 && e.ta.kd >= e.ta.ls) sm = (size_t)e.ta.dsoff * sizeof(float) + sizeof(float) * (size_t)e.ta.dld;
      tail_smem = std::max(tail_smem, sm);
    }
    const int cap = batch_sweep_capacity<S>();
    sweep_items.resize(maxlt);
    plain_items.resize(maxlt);
    restrict_items.resize(maxlt);
    prolong_items.resize(maxlt);
    sweep_items_n.assign(maxlt, 0);
    sweep_ctas.assign(maxlt, 0);
    plain_ctas.assign(maxlt, 0);
    restrict_ctas.assign(maxlt, 0);
    prolong_ctas.assign(maxlt, 0);
    auto blocks_for = [&](i64 threads) { return (int)std::max<i64>(1, std::min<i64>(ceil_div(threads, 256), sms * 8)); };
    for (int l = 0; l < maxlt; ++l) {
      std::vector<BatchItem> sw, pl, re, pr;
      int c0 = 0, p0 = 0, r0 = 0, q0 = 0;
      for (const auto& e : v) {
        if (l >= e.lt) continue;
        BatchItem it{};
        it.lv = e.lv[l];
        it.dim = e.dim;
        it.G = e.G[l];
        it.cta0 = c0;
        it.nb = e.lv[l].R;
        sw.push_back(it);
        c0 += it.nb;
        it.cta0 = p0;
        it.nb = blocks_for((i64)e.lv[l].nv * it.G);
        pl.push_back(it);
        p0 += it.nb;
        it.cta0 = r0;
        it.nb = blocks_for(e.lv[l].nvc);
        re.push_back(it);
        r0 += it.nb;
        it.cta0 = q0;
        it.nb = blocks_for(e.lv[l].nv);
        pr.push_back(it);
        q0 += it.nb;
      }
      VASMG_CHECK(c0 <= cap, VASMG_ERR_UNSUPPORTED, "the batch's regions do not fit the device at once");
      auto up = [&](DevBuf<BatchItem>& d, const std::vector<BatchItem>& h) {
        d.alloc((i64)std::max<size_t>(1, h.size()), s);
        if (!h.empty()) d.upload(h.data(), (i64)h.size());
      };
      up(sweep_items[l], sw);
      up(plain_items[l], pl);
      up(restrict_items[l], re);
      up(prolong_items[l], pr);
      sweep_items_n[l] = (int)sw.size();
      sweep_ctas[l] = c0;
      plain_ctas[l] = p0;
      restrict_ctas[l] = r0;
      prolong_ctas[l] = q0;
    }
    std::vector<TailArgs<float>> ta(n);
    std::vector<int> dims(n);
    std::vector<CGB> cgh(n);
    for (int i = 0; i < n; ++i) {
      ta[i] = v[i].ta;
      dims[i] = v[i].dim;
      CGB& m = cgh[i];
      m.a = v[i].cga;
      m.a.cond = 0;
      m.b0 = v[i].lv[0].b;
      m.z = v[i].lv[0].x;
      m.F = v[i].Fbuf;
      m.Uout = v[i].Ubuf;
      m.dim = v[i].dim;
      m.cg_blocks = v[i].cg_blocks;
      m.spmv_blocks = v[i].spmv_blocks;
      cg_grid = std::max(cg_grid, m.cg_blocks);
      spmv_grid = std::max(spmv_grid, m.spmv_blocks);
    }
    targs.alloc(n, s);
    targs.upload(ta.data(), n);
    tdims.alloc(n, s);
    tdims.upload(dims.data(), n);
    cg.alloc(n, s);
    cg.upload(cgh.data(), n);
    ctl.alloc(2, s);
    ctl.zero();
    abort_flag.alloc(1, s);
    abort_flag.zero();
    VASMG_CHECK(tail_smem <= (size_t)TAIL_SMEM_MAX, VASMG_ERR_UNSUPPORTED, "tail levels too large for shared memory");
    VASMG_CUDA(cudaFuncSetAttribute(tailb_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, TAIL_SMEM_MAX));
    if (nct > 8 && cudaFuncSetAttribute(tailb_kernel<S>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                       cudaSuccess)
      nct = 8;
    cudaGetLastError();
    // one cluster size for all tails (a row's arithmetic does not depend on
    // it): the largest the handles use that the device can hold
    while (nct > 1) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(nct);
      cfg.blockDim = dim3(TAIL_THREADS);
      cfg.dynamicSmemBytes = tail_smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = nct;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, tailb_kernel<S>, &cfg) == cudaSuccess && nclusters > 0) break;
      cudaGetLastError();
      nct /= 2;
    }
  }

  template <typename K>
  void coop(K kern, int grid, int l) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(DFM_THREADS);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const BatchItem* items = sweep_items[l].get();
    const int ni = sweep_items_n[l];
    int* ab = abort_flag.get();
    VASMG_CUDA(cudaLaunchKernelEx(&cfg, kern, items, ni, ab));
    ++launches;
  }
  void vcycle() {
    for (int l = 0; l < maxlt; ++l) {
      if (!sweep_items_n[l]) continue;
      coop(sweepb_kernel<S, 0>, sweep_ctas[l], l);
      residualb_kernel<S><<<plain_ctas[l], DFM_THREADS, 0, s>>>(plain_items[l].get(), sweep_items_n[l]);
      transferb_kernel<0><<<restrict_ctas[l], DFM_THREADS, 0, s>>>(restrict_items[l].get(), sweep_items_n[l]);
      launches += 2;
    }
    {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(nct * n);
      cfg.blockDim = dim3(TAIL_THREADS);
      cfg.dynamicSmemBytes = tail_smem;
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = nct;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      const TailArgs<float>* tp = targs.get();
      const int* dp = tdims.get();
      VASMG_CUDA(cudaLaunchKernelEx(&cfg, tailb_kernel<S>, tp, dp));
      ++launches;
    }
    for (int l = maxlt - 1; l >= 0; --l) {
      if (!sweep_items_n[l]) continue;
      transferb_kernel<1><<<prolong_ctas[l], DFM_THREADS, 0, s>>>(prolong_items[l].get(), sweep_items_n[l]);
      ++launches;
      coop(sweepb_kernel<S, 1>, sweep_ctas[l], l);
    }
  }
  template <bool COND>
  void body() {
    vcycle();
    const dim3 gc(cg_grid, n), gs(spmv_grid, n);
    cgb_rz_kernel<<<gc, CG_THREADS, 0, s>>>(cg.get());
    cgb_pupdate_kernel<<<gc, CG_THREADS, 0, s>>>(cg.get());
    cgb_spmv_kernel<<<gs, CG_THREADS, 0, s>>>(cg.get());
    cgb_update_kernel<<<gc, CG_THREADS, 0, s>>>(cg.get(), abort_flag.get());
    cgb_cond_kernel<COND><<<1, 32, 0, s>>>(cg.get(), n, ctl.get(), max_iters, cond, 1);
    launches += 5;
  }
  // init -> WHILE(any active){ body } -> final, as one graph; false if the
  // conditional graph cannot be built
  bool run_graph() {
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
    bool ok = true;
    cudaGraphConditionalHandle h = 0;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) ok = false;
    cudaGraph_t out = nullptr;
    cudaGraphNode_t last = nullptr, wnode = nullptr;
    if (ok) {
      cond = (unsigned long long)h;
      ok = cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        cgb_init_kernel<<<dim3(cg_grid, n), CG_THREADS, 0, s>>>(cg.get());
        cgb_cond_kernel<true><<<1, 32, 0, s>>>(cg.get(), n, ctl.get(), max_iters, cond, 0);
        ok = cudaStreamEndCapture(s, &out) == cudaSuccess;
      }
    }
    if (ok) {
      size_t nn = 0;
      ok = cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn == 2;
      cudaGraphNode_t nodes[2];
      if (ok) ok = cudaGraphGetNodes(g, nodes, &nn) == cudaSuccess;
      if (ok) {
        cudaKernelNodeParams kp = {};
        ok = cudaGraphKernelNodeGetParams(nodes[1], &kp) == cudaSuccess;
        last = (ok && kp.func == (void*)cgb_cond_kernel<true>) ? nodes[1] : nodes[0];
      }
    }
    if (ok) {
      cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      ok = cudaGraphAddNode(&wnode, g, &last, nullptr, 1, &np) == cudaSuccess;
      if (ok) {
        cudaGraph_t bodyg = np.conditional.phGraph_out[0];
        ok = cudaStreamBeginCaptureToGraph(s, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
          try {
            body<true>();
          } catch (...) {
            ok = false;
          }
          ok = (cudaStreamEndCapture(s, &out) == cudaSuccess) && ok;
        }
      }
    }
    if (ok) {
      ok = cudaStreamBeginCaptureToGraph(s, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        cgb_final_kernel<<<dim3(cg_grid, n), CG_THREADS, 0, s>>>(cg.get());
        ok = cudaStreamEndCapture(s, &out) == cudaSuccess;
      }
    }
    cudaGraphExec_t ex = nullptr;
    if (ok && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
      ex = nullptr;
      ok = false;
    }
    cudaGraphDestroy(g);
    cudaGetLastError();
    cond = 0;
    if (!ok) return false;
    const cudaError_t e = cudaGraphLaunch(ex, s);
    cudaStreamSynchronize(s);
    cudaGraphExecDestroy(ex);
    VASMG_CUDA(e);
    return true;
  }
  // the same with a host loop over per-iteration launches
  void run_host() {
    cgb_init_kernel<<<dim3(cg_grid, n), CG_THREADS, 0, s>>>(cg.get());
    cgb_cond_kernel<false><<<1, 32, 0, s>>>(cg.get(), n, ctl.get(), max_iters, 0, 0);
    check_launch("cgb_init");
    int h[2] = {0, 1};
    VASMG_CUDA(cudaMemcpyAsync(h, ctl.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
    VASMG_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; h[1] && b <= max_iters + 2; ++b) {
      body<false>();
      VASMG_CUDA(cudaMemcpyAsync(h, ctl.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
      VASMG_CUDA(cudaStreamSynchronize(s));
    }
    cgb_final_kernel<<<dim3(cg_grid, n), CG_THREADS, 0, s>>>(cg.get());
    check_launch("cgb_final");
  }
};

template <typename S>
int batch_solve(const std::vector<EngineView<float>>& views, cudaStream_t s, const double* const* F,
                double* const* U, double tol, vasmg_stats* st, i64* launches) {
  const int n = (int)views.size();
  if (n == 0) return VASMG_OK;
  BatchRun<S> br(views, s);
  for (int i = 0; i < n; ++i) {
    const EngineView<float>& e = views[i];
    Scalars init{};
    init.tol = tol;
    init.max_iters = e.max_iters;
    VASMG_CUDA(cudaMemcpyAsync(e.cga.sc, &init, sizeof(Scalars), cudaMemcpyHostToDevice, s));
    VASMG_CUDA(cudaMemcpyAsync(e.Fbuf, F[i], sizeof(double) * e.nv[0] * e.dim, cudaMemcpyDefault, s));
  }
  bool graph = true;
  for (const auto& e : views) graph = graph && e.use_graph;
  i64 iter_launches = 0;
  {
    // one body's launches, counted by a dry run of the host loop's bookkeeping
    const i64 before = br.launches;
    if (!(graph && br.run_graph())) {
      br.launches = before;
      br.run_host();
    }
    iter_launches = br.launches - before;
  }
  std::vector<Scalars> hs(n);
  int ctlh[2] = {0, 0};
  for (int i = 0; i < n; ++i)
    VASMG_CUDA(cudaMemcpyAsync(&hs[i], views[i].cga.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  VASMG_CUDA(cudaMemcpyAsync(ctlh, br.ctl.get(), sizeof(ctlh), cudaMemcpyDeviceToHost, s));
  int ab = 0;
  VASMG_CUDA(cudaMemcpyAsync(&ab, br.abort_flag.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  for (int i = 0; i < n; ++i)
    VASMG_CUDA(cudaMemcpyAsync(U[i], views[i].Ubuf, sizeof(double) * views[i].nv[0] * views[i].dim,
                               cudaMemcpyDefault, s));
  VASMG_CUDA(cudaStreamSynchronize(s));
  // graph path: the body captured once, run ctl[0] times (+ init, condition, final)
  if (launches) *launches = graph ? 3 + iter_launches * (i64)ctlh[0] : iter_launches + 3;
  int worst = VASMG_OK;
  for (int i = 0; i < n; ++i) {
    int rc = hs[i].status;
    if (ab) rc = VASMG_ERR_TIMEOUT;
    if (st) {
      st[i].iterations = hs[i].iter;
      st[i].rel_res = hs[i].relres;
      st[i].n_levels = views[i].L;
      if (st[i].res_history && st[i].res_history_cap > 0) {
        const int kk = std::min(st[i].res_history_cap, std::min(hs[i].iter, views[i].max_iters));
        if (kk > 0)
          VASMG_CUDA(cudaMemcpy(st[i].res_history, views[i].cga.hist, sizeof(double) * kk, cudaMemcpyDeviceToHost));
      }
    }
    if (rc < 0) worst = std::min(worst, rc);
    else if (worst >= 0) worst = std::max(worst, rc);
  }
  return worst;
}

template int batch_solve<float>(const std::vector<EngineView<float>>&, cudaStream_t, const double* const*,
                                double* const*, double, vasmg_stats*, i64*);
template int batch_solve<__nv_bfloat16>(const std::vector<EngineView<float>>&, cudaStream_t, const double* const*,
                                        double* const*, double, vasmg_stats*, i64*);
template int batch_sweep_capacity<float>();
template int batch_sweep_capacity<__nv_bfloat16>();

template <int D, typename S>
MultiBase* make_multi(const EngineView<float>& v) {
  return new MultiEngine<D, S>(v);
}

template MultiBase* make_multi<2, float>(const EngineView<float>&);
template MultiBase* make_multi<2, __nv_bfloat16>(const EngineView<float>&);
template MultiBase* make_multi<3, float>(const EngineView<float>&);
template MultiBase* make_multi<3, __nv_bfloat16>(const EngineView<float>&);

}  // namespace vasmg
