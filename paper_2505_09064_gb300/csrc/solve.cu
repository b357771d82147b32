// The hot path: one PCG iteration (Alg. 2) preconditioned by one V-cycle
// (Alg. 3, recursive) of V-ASMG.
//
// Outer CG, FP64, level-0 solve order:
//   spmv_dot     q = A p (diagonal + off-diagonal planes), p.q, alpha = rho / p.q
//   cg_update    U += alpha p, r -= alpha q, ||r||, stop test ||r||/||F|| < tol
//                (Sec. 5 item (3)), b_0 = r cast to the V-cycle precision
//   rz_dot       rho_new = r.z, beta = rho_new / rho
//   p_update     p = z + beta p
// Reductions are deterministic: every block writes one partial, and the last
// block to finish sums the partials in index order.
//
// V-cycle, level by level (precision V, values stored as S):
//   pre-smooth   one forward multicolour block Gauss-Seidel sweep from a zero
//                initial guess: x_i = D_ii^{-1} (b_i - sum_{j of an earlier
//                colour} A_ij x_j) -- with a zero start the later colours
//                contribute nothing, so only the "lower" part of each row
//                (columns of earlier colours come first) is read;
//   residual     r_i = - sum_{j of a later colour} A_ij x_j: after that sweep
//                b_i - A_ii x_i - sum_lower A_ij x_j is exactly zero, so only the
//                "upper" part is read (pre-smooth + residual = one pass over A);
//   restrict     b_{l+1} = R r_l with R = P^T (eq. (R)), gathered row-wise;
//   coarsest     A_L e = b by the FP64 Cholesky factor (Sec. 3, Step 2.3);
//   prolong      x_l += P e_{l+1} (masked at dead dofs);
//   post-smooth  one backward sweep (colours in reverse order) with full rows.
// Levels with at most TAIL_NV vertices run in a single one-CTA kernel.
//
// Every loop of the solve is captured in one CUDA graph with a conditional
// WHILE node, so a solve is one graph launch (no host round trip per
// iteration); without graph support the host launches the per-iteration body
// and reads the stop flag.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace vasmg {

constexpr int TAIL_NV = 4096;
constexpr int TAIL_THREADS = 1024;
constexpr int TAIL_G = 8;
constexpr int MAX_LEVELS = 48;
constexpr int CG_THREADS = 256;

struct Scalars {
  double rho, pq, alpha, beta, rr, res0, relres, tol;
  int iter, max_iters, done, status, first, bodies;
  unsigned int cnt[4];
};

// ------------------------------------------------------------------ loads

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

template <typename V>
struct LV {
  int nv;
  long long nnz;
  const int* rp;
  const int* ci;
  const int* sp;
  const void* off;        // planes [d*d][nnz] of S
  const V* dinv;          // planes [d*d][nv]
  const uint8_t* dead;    // per vertex, bit a = component a removed
  V* x;
  V* b;
  V* r;
  // transfer to level l+1
  const int* prp;
  const int* pci;
  const V* pw;
  const int* rrp;
  const int* rci;
  const V* rw;
};

template <int D>
__device__ __forceinline__ double pick(const double (&a)[D], int i) {
  return D == 2 ? (i == 0 ? a[0] : a[1]) : (i == 0 ? a[0] : (i == 1 ? a[1] : a[D - 1]));
}
template <int D>
__device__ __forceinline__ float pick(const float (&a)[D], int i) {
  return D == 2 ? (i == 0 ? a[0] : a[1]) : (i == 0 ? a[0] : (i == 1 ? a[1] : a[D - 1]));
}

// One row of a sweep / residual by a group of G lanes.
// MODE 0: x_i = Dinv (b_i - lower part), MODE 1: x_i = Dinv (b_i - all
// off-diagonal blocks), MODE 2: r_i = -(upper part).
template <int D, int G, typename V, typename S, int MODE>
__device__ __forceinline__ void row_pass(const LV<V>& L, int row, bool valid, int lane) {
  int k0 = 0, k1 = 0;
  if (valid) {
    k0 = MODE == 2 ? __ldg(L.sp + row) : __ldg(L.rp + row);
    k1 = MODE == 0 ? __ldg(L.sp + row) : __ldg(L.rp + row + 1);
  }
  const S* off = (const S*)L.off;
  V acc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) acc[a] = V(0);
  for (int k = k0 + lane; k < k1; k += G) {
    const int j = __ldg(L.ci + k);
    V xj[D];
#pragma unroll
    for (int bb = 0; bb < D; ++bb) xj[bb] = L.x[(long long)j * D + bb];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int bb = 0; bb < D; ++bb) acc[a] += ldv<V, S>(off + (long long)(a * D + bb) * L.nnz + k) * xj[bb];
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o, G);
  if (!valid || lane >= D) return;
  if (MODE == 2) {
    L.r[(long long)row * D + lane] = -pick<D>(acc, lane);
  } else {
    V s = V(0);
#pragma unroll
    for (int bb = 0; bb < D; ++bb)
      s += __ldg(L.dinv + (long long)(lane * D + bb) * L.nv + row) * (L.b[(long long)row * D + bb] - acc[bb]);
    L.x[(long long)row * D + lane] = s;
  }
}

template <int D, int G, typename V, typename S, int MODE>
__global__ void __launch_bounds__(256) colour_kernel(LV<V> L, int row0, int row1) {
  const int gid = (int)((blockIdx.x * blockDim.x + threadIdx.x) / G);
  const int lane = threadIdx.x & (G - 1);
  const int row = row0 + gid;
  row_pass<D, G, V, S, MODE>(L, row, row < row1, lane);
}

template <int D, typename V>
__device__ __forceinline__ void restrict_row(const LV<V>& L, const LV<V>& C, int I) {
  V acc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) acc[a] = V(0);
  for (int t = __ldg(L.rrp + I); t < __ldg(L.rrp + I + 1); ++t) {
    const int i = __ldg(L.rci + t);
    const V w = __ldg(L.rw + t);
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] += w * L.r[(long long)i * D + a];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) C.b[(long long)I * D + a] = acc[a];
}

template <int D, typename V>
__device__ __forceinline__ void prolong_row(const LV<V>& L, const LV<V>& C, int i) {
  V acc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) acc[a] = V(0);
  for (int t = __ldg(L.prp + i); t < __ldg(L.prp + i + 1); ++t) {
    const int J = __ldg(L.pci + t);
    const V w = __ldg(L.pw + t);
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] += w * C.x[(long long)J * D + a];
  }
  const uint8_t dm = __ldg(L.dead + i);
#pragma unroll
  for (int a = 0; a < D; ++a)
    if (!((dm >> a) & 1)) L.x[(long long)i * D + a] += acc[a];
}

template <int D, typename V>
__global__ void __launch_bounds__(256) restrict_kernel(LV<V> L, LV<V> C) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < C.nv) restrict_row<D, V>(L, C, I);
}

template <int D, typename V>
__global__ void __launch_bounds__(256) prolong_kernel(LV<V> L, LV<V> C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L.nv) prolong_row<D, V>(L, C, i);
}

// ------------------------------------------------------------------ coarsest solve and tail

struct CoarseArgs {
  const double* chol;      // n x n lower factor, canonical dof order
  const uint8_t* drop;
  const int* perm;         // solve index -> canonical vertex (coarsest level)
  double* y;               // scratch [n]
  int n, d;
};

// Forward / backward substitution with the Cholesky factor, by one warp.
template <typename V>
__device__ void coarse_solve_warp(const CoarseArgs& A, const V* b, V* x) {
  const int lane = threadIdx.x & 31;
  const int n = A.n, d = A.d;
  for (int t = lane; t < n; t += 32) {
    const int r = t / d, a = t - r * d;
    A.y[(long long)__ldg(A.perm + r) * d + a] = (double)b[t];
  }
  __syncwarp();
  for (int j = 0; j < n; ++j) {
    const double ljj = A.chol[(long long)j * n + j];
    const double yj = A.drop[j] ? 0.0 : A.y[j] / ljj;
    __syncwarp();
    if (lane == 0) A.y[j] = yj;
    for (int i = j + 1 + lane; i < n; i += 32) A.y[i] -= A.chol[(long long)i * n + j] * yj;
    __syncwarp();
  }
  for (int j = n - 1; j >= 0; --j) {
    const double ljj = A.chol[(long long)j * n + j];
    const double xj = A.drop[j] ? 0.0 : A.y[j] / ljj;
    __syncwarp();
    if (lane == 0) A.y[j] = xj;
    for (int i = lane; i < j; i += 32) A.y[i] -= A.chol[(long long)j * n + i] * xj;
    __syncwarp();
  }
  for (int t = lane; t < n; t += 32) {
    const int r = t / d, a = t - r * d;
    x[t] = (V)A.y[(long long)__ldg(A.perm + r) * d + a];
  }
}

template <typename V>
__global__ void coarse_kernel(CoarseArgs A, const V* b, V* x) {
  if (threadIdx.x < 32) coarse_solve_warp<V>(A, b, x);
}

template <typename V>
struct TailArgs {
  int l0, L;                     // levels l0..L handled here, L = coarsest
  LV<V> lv[MAX_LEVELS];
  const int* cs[MAX_LEVELS];     // colour starts per level (device)
  int ncol[MAX_LEVELS];
  CoarseArgs co;
};

// The V-cycle of all small levels in one CTA (phases separated by
// __syncthreads; every group runs the same number of loop trips so the
// sub-warp shuffles stay converged).
template <int D, typename V, typename S>
__global__ void __launch_bounds__(TAIL_THREADS) tail_kernel(const TailArgs<V>* __restrict__ T) {
  constexpr int G = TAIL_G;
  const int g = threadIdx.x / G, lane = threadIdx.x & (G - 1), ng = blockDim.x / G;
  const int l0 = T->l0, Lc = T->L;
  for (int l = l0; l < Lc; ++l) {
    const LV<V>& L = T->lv[l];
    const int* cs = T->cs[l];
    for (int c = 0; c < T->ncol[l]; ++c) {
      const int r0 = cs[c], r1 = cs[c + 1];
      for (int base = r0; base < r1; base += ng) row_pass<D, G, V, S, 0>(L, base + g, base + g < r1, lane);
      __syncthreads();
    }
    for (int base = 0; base < L.nv; base += ng) row_pass<D, G, V, S, 2>(L, base + g, base + g < L.nv, lane);
    __syncthreads();
    const LV<V>& C = T->lv[l + 1];
    for (int I = threadIdx.x; I < C.nv; I += blockDim.x) restrict_row<D, V>(L, C, I);
    __syncthreads();
  }
  if (threadIdx.x < 32) coarse_solve_warp<V>(T->co, T->lv[Lc].b, T->lv[Lc].x);
  __syncthreads();
  for (int l = Lc - 1; l >= l0; --l) {
    const LV<V>& L = T->lv[l];
    const LV<V>& C = T->lv[l + 1];
    for (int i = threadIdx.x; i < L.nv; i += blockDim.x) prolong_row<D, V>(L, C, i);
    __syncthreads();
    const int* cs = T->cs[l];
    for (int c = T->ncol[l] - 1; c >= 0; --c) {
      const int r0 = cs[c], r1 = cs[c + 1];
      for (int base = r0; base < r1; base += ng) row_pass<D, G, V, S, 1>(L, base + g, base + g < r1, lane);
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ outer CG (FP64)

struct CGArgs {
  int nv;
  long long nnz;
  const int* rp;
  const int* ci;
  const double* off;       // planes [d*d][nnz]
  const double* diag;      // planes [d*d][nv]
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
// the ordered sum of all partials in *total (thread 0).
__device__ __forceinline__ bool last_block_sum(double v, double* part, unsigned int* counter, double* total) {
  __shared__ double sh[32];
  __shared__ bool is_last;
  const double b = block_sum(v, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = b;
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(part + i);
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) {
    *total = tot;
    *counter = 0u;
  }
  return true;
}

__device__ __forceinline__ void set_cond(unsigned long long h, unsigned int v) {
  if (h) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
}

// r = F - A u_D at free dofs (0 at Dirichlet dofs), gathered into solve order;
// U = p = 0; res0 = ||r||; b_0 = (V) r.
template <int D, typename V>
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
    s->first = 1;
    s->status = 0;
    s->done = (s->res0 == 0.0) ? 1 : 0;
    if (s->done) s->relres = 0.0;
    set_cond(a.cond, s->done ? 0u : 1u);
  }
}

// rho_new = r . z; beta = rho_new / rho (0 on the first iteration)
template <int D, typename V>
__global__ void __launch_bounds__(CG_THREADS) rz_kernel(CGArgs a, const V* __restrict__ z) {
  double acc = 0.0;
  const long long n = (long long)a.nv * D;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    acc += a.r[t] * (double)z[t];
  // hard bound on loop bodies, independent of the reductions below: the
  // device-side WHILE loop can never run more than max_iters + 2 bodies
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Scalars* s = a.sc;
    s->bodies += 1;
    if (s->bodies > s->max_iters + 2) {
      s->done = 1;
      s->status = VASMG_ERR_TIMEOUT;
      set_cond(a.cond, 0u);
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
    a.p[t] = (double)z[t] + beta * a.p[t];
}

// q = A p (diagonal planes + off-diagonal planes), p.q, alpha = rho / p.q.
template <int D, int G>
__global__ void __launch_bounds__(CG_THREADS) spmv_dot_kernel(CGArgs a, int with_dot) {
  const int lane = threadIdx.x & (G - 1);
  const int gpb = CG_THREADS / G;
  double dot = 0.0;
  for (int base = blockIdx.x * gpb; base < a.nv; base += gridDim.x * gpb) {
    const int row = base + (int)threadIdx.x / G;
    const bool valid = row < a.nv;
    int k0 = 0, k1 = 0;
    if (valid) {
      k0 = __ldg(a.rp + row);
      k1 = __ldg(a.rp + row + 1);
    }
    double acc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = 0.0;
    if (valid && lane == 0) {
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int bb = 0; bb < D; ++bb)
          acc[c] += __ldg(a.diag + (long long)(c * D + bb) * a.nv + row) * a.p[(long long)row * D + bb];
    }
    for (int k = k0 + lane; k < k1; k += G) {
      const int j = __ldg(a.ci + k);
      double pj[D];
#pragma unroll
      for (int bb = 0; bb < D; ++bb) pj[bb] = a.p[(long long)j * D + bb];
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int bb = 0; bb < D; ++bb) acc[c] += __ldg(a.off + (long long)(c * D + bb) * a.nnz + k) * pj[bb];
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o, G);
    if (valid && lane < D) {
      const double qv = pick<D>(acc, lane);
      a.q[(long long)row * D + lane] = qv;
      dot += qv * a.p[(long long)row * D + lane];
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
      set_cond(a.cond, 0u);
    } else {
      s->alpha = s->rho / tot;
    }
  }
}

// U += alpha p; r -= alpha q; ||r||; stop test; b_0 = (V) r.
template <int D, typename V>
__global__ void __launch_bounds__(CG_THREADS) cg_update_kernel(CGArgs a, V* b0) {
  if (a.sc->done) return;  // breakdown in spmv_dot
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
    if (s->relres < s->tol) {
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
    set_cond(a.cond, s->done ? 0u : 1u);
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

// ------------------------------------------------------------------ conversions for vasmg_apply

template <typename V>
__global__ void to_solve_kernel(const double* __restrict__ in, V* __restrict__ out, const int* __restrict__ perm,
                                long long nv, int d) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nv * d; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / d;
    out[t] = (V)in[(long long)perm[r] * d + (t - r * d)];
  }
}
template <typename V>
__global__ void from_solve_kernel(const V* __restrict__ in, double* __restrict__ out, const int* __restrict__ perm,
                                  long long nv, int d) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nv * d; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / d;
    out[(long long)perm[r] * d + (t - r * d)] = (double)in[t];
  }
}

// ------------------------------------------------------------------ engine

struct EngineBase {
  virtual ~EngineBase() {}
  virtual int solve(Ctx& c, const double* F, double* U, double tol, vasmg_stats* st) = 0;
  virtual void apply(Ctx& c, int op, int level, const double* x, double* y) = 0;
  virtual double time(Ctx& c, int which, int level, int reps, double* bytes) = 0;
};

static int pick_G(double avg) {
  if (avg <= 6.0) return 4;
  if (avg <= 12.0) return 8;
  if (avg <= 24.0) return 16;
  return 32;
}

template <int D, typename V, typename S>
struct Engine : EngineBase {
  Ctx* c = nullptr;
  int L = 0;       // number of levels
  int lt = 0;      // first tail level
  std::vector<LV<V>> lv;
  std::vector<int> G;
  std::vector<DevBuf<int32_t>> cs_dev;
  DevBuf<TailArgs<V>> tail;
  DevBuf<double> coarse_y;
  // CG
  DevBuf<double> U, r, p, q, part, hist, Fbuf, Ubuf;
  DevBuf<Scalars> sc;
  Scalars* host_sc = nullptr;
  CGArgs cga{};
  int cg_blocks = 0, spmv_blocks = 0, G0 = 8;
  CoarseArgs co{};
  // graphs
  cudaGraphExec_t exec_while = nullptr;
  cudaGraphExec_t exec_body = nullptr;
  i64 launches_body = 0, launches_outer = 0;
  i64 launch_counter = 0;

  explicit Engine(Ctx& ctx) : c(&ctx) { build(); }
  ~Engine() override {
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

  void build() {
    cudaStream_t s = c->stream;
    L = (int)c->S.size();
    VASMG_CHECK(L <= MAX_LEVELS, VASMG_ERR_UNSUPPORTED, "too many levels");
    lv.resize(L);
    G.resize(L);
    cs_dev.resize(L);
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
      v.prp = sl.prp.get();
      v.pci = sl.pci.get();
      v.pw = pw_ptr(sl);
      v.rrp = sl.rrp.get();
      v.rci = sl.rci.get();
      v.rw = rw_ptr(sl);
      G[l] = pick_G(sl.nv > 0 ? (double)sl.nnz / (double)sl.nv : 1.0);
    }
    lt = L - 1;
    while (lt > 0 && c->S[lt - 1].nv <= TAIL_NV) --lt;
    // coarsest
    coarse_y.alloc(c->nc, s);
    co.chol = c->chol.get();
    co.drop = c->chol_drop.get();
    co.perm = c->S[L - 1].perm.get();
    co.y = coarse_y.get();
    co.n = (int)c->nc;
    co.d = D;
    {
      std::vector<char> hbuf(sizeof(TailArgs<V>), 0);
      TailArgs<V>* ta = (TailArgs<V>*)hbuf.data();
      ta->l0 = lt;
      ta->L = L - 1;
      for (int l = 0; l < L; ++l) {
        ta->lv[l] = lv[l];
        ta->cs[l] = cs_dev[l].get();
        ta->ncol[l] = c->S[l].ncol;
      }
      ta->co = co;
      tail.alloc(1, s);
      VASMG_CUDA(cudaMemcpyAsync(tail.get(), hbuf.data(), sizeof(TailArgs<V>), cudaMemcpyHostToDevice, s));
    }
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
    int dev = 0, sms = 0;
    VASMG_CUDA(cudaGetDevice(&dev));
    VASMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cg_blocks = (int)std::max<i64>(1, std::min<i64>((i64)sms * 8, ceil_div(n, CG_THREADS)));
    G0 = pick_G((double)s0.nnz / std::max<i64>(1, s0.nv) + 1.0);
    spmv_blocks = (int)std::max<i64>(1, std::min<i64>((i64)sms * 8, ceil_div(s0.nv, CG_THREADS / G0)));
    part.alloc(std::max(cg_blocks, spmv_blocks), s);
    hist.alloc(std::max(1, c->max_iters), s);
    sc.alloc(1, s);
    sc.zero();
    VASMG_CUDA(cudaMallocHost((void**)&host_sc, sizeof(Scalars)));
    cga.nv = (int)s0.nv;
    cga.nnz = s0.nnz;
    cga.rp = s0.rp.get();
    cga.ci = s0.ci.get();
    cga.off = s0.off64.get();
    cga.diag = s0.diag64.get();
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
    VASMG_CUDA(cudaStreamSynchronize(s));
  }

  // ---------------------------------------------------------------- launches
  template <int MODE>
  void colour_launch(int l, int row0, int row1, cudaStream_t s) {
    if (row1 <= row0) return;
    const int g = G[l];
    const i64 threads = (i64)(row1 - row0) * g;
    const int blocks = (int)ceil_div(threads, 256);
    switch (g) {
      case 4: colour_kernel<D, 4, V, S, MODE><<<blocks, 256, 0, s>>>(lv[l], row0, row1); break;
      case 8: colour_kernel<D, 8, V, S, MODE><<<blocks, 256, 0, s>>>(lv[l], row0, row1); break;
      case 16: colour_kernel<D, 16, V, S, MODE><<<blocks, 256, 0, s>>>(lv[l], row0, row1); break;
      default: colour_kernel<D, 32, V, S, MODE><<<blocks, 256, 0, s>>>(lv[l], row0, row1); break;
    }
    ++launch_counter;
  }
  void sweep_fwd_zero(int l, cudaStream_t s) {
    const auto& cs = c->S[l].cs;
    for (int col = 0; col < c->S[l].ncol; ++col) colour_launch<0>(l, cs[col], cs[col + 1], s);
  }
  void sweep_bwd(int l, cudaStream_t s) {
    const auto& cs = c->S[l].cs;
    for (int col = c->S[l].ncol - 1; col >= 0; --col) colour_launch<1>(l, cs[col], cs[col + 1], s);
  }
  void residual(int l, cudaStream_t s) { colour_launch<2>(l, 0, lv[l].nv, s); }
  void restrict_to(int l, cudaStream_t s) {
    restrict_kernel<D, V><<<grid_for(lv[l + 1].nv, 256), 256, 0, s>>>(lv[l], lv[l + 1]);
    ++launch_counter;
  }
  void prolong_from(int l, cudaStream_t s) {
    prolong_kernel<D, V><<<grid_for(lv[l].nv, 256), 256, 0, s>>>(lv[l], lv[l + 1]);
    ++launch_counter;
  }
  void tail_launch(cudaStream_t s) {
    tail_kernel<D, V, S><<<1, TAIL_THREADS, 0, s>>>(tail.get());
    ++launch_counter;
  }
  // V-cycle from level l0 (b_{l0} set, result in x_{l0}).
  void vcycle(int l0, cudaStream_t s) {
    if (l0 >= lt) {
      if (l0 == lt) {
        tail_launch(s);
        return;
      }
      // a V-cycle starting inside the tail range: run per level for exactness
      for (int l = l0; l < L - 1; ++l) {
        sweep_fwd_zero(l, s);
        residual(l, s);
        restrict_to(l, s);
      }
      coarse_kernel<V><<<1, 32, 0, s>>>(co, lv[L - 1].b, lv[L - 1].x);
      ++launch_counter;
      for (int l = L - 2; l >= l0; --l) {
        prolong_from(l, s);
        sweep_bwd(l, s);
      }
      return;
    }
    for (int l = l0; l < lt; ++l) {
      sweep_fwd_zero(l, s);
      residual(l, s);
      restrict_to(l, s);
    }
    tail_launch(s);
    for (int l = lt - 1; l >= l0; --l) {
      prolong_from(l, s);
      sweep_bwd(l, s);
    }
  }

  void spmv(cudaStream_t s, int with_dot) {
    switch (G0) {
      case 4: spmv_dot_kernel<D, 4><<<spmv_blocks, CG_THREADS, 0, s>>>(cga, with_dot); break;
      case 8: spmv_dot_kernel<D, 8><<<spmv_blocks, CG_THREADS, 0, s>>>(cga, with_dot); break;
      case 16: spmv_dot_kernel<D, 16><<<spmv_blocks, CG_THREADS, 0, s>>>(cga, with_dot); break;
      default: spmv_dot_kernel<D, 32><<<spmv_blocks, CG_THREADS, 0, s>>>(cga, with_dot); break;
    }
    ++launch_counter;
  }

  // One PCG iteration, rotated so the stop test ends it: z = M r; rho, beta;
  // p = z + beta p; q = A p, alpha; U, r update + stop test.
  void body(cudaStream_t s) {
    V* z = lv[0].x;
    vcycle(0, s);
    rz_kernel<D, V><<<cg_blocks, CG_THREADS, 0, s>>>(cga, z);
    p_update_kernel<D, V><<<cg_blocks, CG_THREADS, 0, s>>>(cga, z);
    spmv(s, 1);
    cg_update_kernel<D, V><<<cg_blocks, CG_THREADS, 0, s>>>(cga, lv[0].b);
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
        cg_init_kernel<D, V><<<cg_blocks, CG_THREADS, 0, s>>>(cga, Fbuf.get(), lv[0].b);
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
          body(s);
          ok = cudaStreamEndCapture(s, &out) == cudaSuccess;
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
    body(s);
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
    i64 launches = 0;
    if (exec_while) {
      VASMG_CUDA(cudaGraphLaunch(exec_while, s));
      VASMG_CUDA(cudaMemcpyAsync(host_sc, sc.get(), sizeof(Scalars), cudaMemcpyDeviceToHost, s));
      VASMG_CUDA(cudaStreamSynchronize(s));
    } else {
      cg_init_kernel<D, V><<<cg_blocks, CG_THREADS, 0, s>>>(cga, Fbuf.get(), lv[0].b);
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
    launches = 2 + launches_body * (i64)iters;
    ctx.last_launches = launches;
    if (st) {
      st->iterations = iters;
      st->rel_res = host_sc->relres;
      st->n_levels = L;
      if (st->res_history && st->res_history_cap > 0) {
        const int k = std::min(st->res_history_cap, std::min(iters, c->max_iters));
        if (k > 0) VASMG_CUDA(cudaMemcpy(st->res_history, hist.get(), sizeof(double) * k, cudaMemcpyDeviceToHost));
      }
    }
    return host_sc->status;
  }

  // ---------------------------------------------------------------- single steps
  void to_solve(const double* x, V* out, int l, cudaStream_t s) {
    to_solve_kernel<V><<<grid_for((i64)lv[l].nv * D, 256), 256, 0, s>>>(x, out, c->S[l].perm.get(), lv[l].nv, D);
  }
  void from_solve(const V* in, double* y, int l, cudaStream_t s) {
    from_solve_kernel<V><<<grid_for((i64)lv[l].nv * D, 256), 256, 0, s>>>(in, y, c->S[l].perm.get(), lv[l].nv, D);
  }

  void apply(Ctx& ctx, int op, int l, const double* x, double* y) override {
    cudaStream_t s = c->stream;
    VASMG_CHECK(l >= 0 && l < L, VASMG_ERR_INVALID_ARG, "level out of range");
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
        to_solve(x, lv[l].b, l, s);
        sweep_fwd_zero(l, s);
        from_solve(lv[l].x, y, l, s);
        break;
      case VASMG_OP_SMOOTH_BWD:
        to_solve(x, lv[l].b, l, s);
        to_solve(y, lv[l].x, l, s);
        sweep_bwd(l, s);
        from_solve(lv[l].x, y, l, s);
        break;
      case VASMG_OP_RESIDUAL:
        to_solve(x, lv[l].b, l, s);
        sweep_fwd_zero(l, s);
        residual(l, s);
        from_solve(lv[l].r, y, l, s);
        break;
      case VASMG_OP_RESTRICT:
        VASMG_CHECK(l + 1 < L, VASMG_ERR_INVALID_ARG, "no coarser level");
        to_solve(x, lv[l].r, l, s);
        restrict_to(l, s);
        from_solve(lv[l + 1].b, y, l + 1, s);
        break;
      case VASMG_OP_PROLONG:
        VASMG_CHECK(l + 1 < L, VASMG_ERR_INVALID_ARG, "no coarser level");
        to_solve(x, lv[l + 1].x, l + 1, s);
        to_solve(y, lv[l].x, l, s);
        prolong_from(l, s);
        from_solve(lv[l].x, y, l, s);
        break;
      case VASMG_OP_COARSE:
        to_solve(x, lv[L - 1].b, L - 1, s);
        coarse_kernel<V><<<1, 32, 0, s>>>(co, lv[L - 1].b, lv[L - 1].x);
        from_solve(lv[L - 1].x, y, L - 1, s);
        break;
      case VASMG_OP_VCYCLE:
        to_solve(x, lv[l].b, l, s);
        vcycle(l, s);
        from_solve(lv[l].x, y, l, s);
        break;
      default:
        throw Error(VASMG_ERR_INVALID_ARG, "unknown op");
    }
    check_launch("apply");
    VASMG_CUDA(cudaStreamSynchronize(s));
    (void)ctx;
  }

  // ---------------------------------------------------------------- timing
  double sweep_bytes(int l) {
    const SolveLevel& sl = c->S[l];
    const double n = (double)sl.nv * D;
    return (double)sl.nnz * (D * D * sizeof(S) + 4.0) + (sl.nv + 1.0) * 4.0 + (double)sl.nv * D * D * sizeof(V) +
           3.0 * n * sizeof(V);
  }
  double spmv_bytes() {
    const SolveLevel& sl = c->S[0];
    const double n = (double)sl.nv * D;
    return (double)sl.nnz * (D * D * 8.0 + 4.0) + (sl.nv + 1.0) * 4.0 + (double)sl.nv * D * D * 8.0 + 2.0 * n * 8.0;
  }
  double vcycle_bytes() {
    double b = 0;
    for (int l = 0; l < L - 1; ++l) {
      const SolveLevel& sl = c->S[l];
      const double n = (double)sl.nv * D;
      // pre-smooth + residual: one pass over the off-diagonal blocks; post-smooth: one pass
      b += 2.0 * ((double)sl.nnz * (D * D * sizeof(S) + 4.0) + (sl.nv + 1.0) * 8.0);
      b += 2.0 * (double)sl.nv * D * D * sizeof(V);     // diagonal inverses, twice
      b += 7.0 * n * sizeof(V);                          // b, x twice each; r write+read; prolong x rmw
      const double pn = (double)c->C[l].pnnz;
      b += 2.0 * pn * (4.0 + sizeof(V)) + 2.0 * (sl.nv + 1.0) * 4.0;  // P and R
    }
    return b;
  }

  double time(Ctx& ctx, int which, int level, int reps, double* bytes) override {
    cudaStream_t s = c->stream;
    cudaEvent_t e0, e1;
    VASMG_CUDA(cudaEventCreate(&e0));
    VASMG_CUDA(cudaEventCreate(&e1));
    auto run = [&]() {
      if (which == VASMG_KERNEL_SPMV64) spmv(s, 0);
      else if (which == VASMG_KERNEL_SWEEP) sweep_bwd(level, s);
      else vcycle(0, s);
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
    *bytes = which == VASMG_KERNEL_SPMV64 ? spmv_bytes() : (which == VASMG_KERNEL_SWEEP ? sweep_bytes(level) : vcycle_bytes());
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

void destroy_solver_state(Ctx& c) {
  delete c.eng;
  c.eng = nullptr;
}

int solve_dev(Ctx& c, const double* F_dev, double* U_dev, double tol, vasmg_stats* st) {
  return c.eng->solve(c, F_dev, U_dev, tol, st);
}

void apply_op(Ctx& c, int op, int level, const double* x_dev, double* y_dev) { c.eng->apply(c, op, level, x_dev, y_dev); }

double time_kernel(Ctx& c, int which, int level, int reps, double* bytes) {
  return c.eng->time(c, which, level, reps, bytes);
}

}  // namespace vasmg
