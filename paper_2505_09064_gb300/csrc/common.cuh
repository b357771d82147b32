// Internal declarations shared by the CUDA sources of libvasmg.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <chrono>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/vasmg.h"

namespace vasmg {

typedef int64_t i64;
typedef uint64_t u64;
typedef uint32_t u32;

// ------------------------------------------------------------------ errors

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define VASMG_CUDA(call)                                                                          \
  do {                                                                                            \
    cudaError_t e__ = (call);                                                                     \
    if (e__ != cudaSuccess) {                                                                     \
      throw ::vasmg::Error(e__ == cudaErrorMemoryAllocation ? VASMG_ERR_OOM : VASMG_ERR_CUDA,    \
                           std::string(#call) + ": " + cudaGetErrorString(e__));                  \
    }                                                                                             \
  } while (0)

#define VASMG_CHECK(cond, code, msg)                   \
  do {                                                 \
    if (!(cond)) throw ::vasmg::Error((code), (msg)); \
  } while (0)

inline void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error(VASMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

inline i64 ceil_div(i64 a, i64 b) { return (a + b - 1) / b; }

// ------------------------------------------------------------------ device memory

// Owning device buffer (stream-ordered allocation on the handle's stream).
template <typename T>
struct DevBuf {
  T* p = nullptr;
  i64 n = 0;
  cudaStream_t s = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; n = o.n; s = o.s;
      o.p = nullptr; o.n = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(i64 count, cudaStream_t stream) {
    release();
    s = stream;
    n = count;
    if (count > 0) VASMG_CUDA(cudaMallocAsync((void**)&p, sizeof(T) * (size_t)count, stream));
  }
  void zero() {
    if (n > 0) VASMG_CUDA(cudaMemsetAsync(p, 0, sizeof(T) * (size_t)n, s));
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  T* get() const { return p; }
  void upload(const T* host, i64 count) {
    VASMG_CUDA(cudaMemcpyAsync(p, host, sizeof(T) * (size_t)count, cudaMemcpyHostToDevice, s));
  }
  std::vector<T> download() const {
    std::vector<T> h((size_t)n);
    if (n > 0) {
      VASMG_CUDA(cudaMemcpyAsync(h.data(), p, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost, s));
      VASMG_CUDA(cudaStreamSynchronize(s));
    }
    return h;
  }
};

template <typename T>
T fetch(const T* dptr, cudaStream_t s) {
  T v;
  VASMG_CUDA(cudaMemcpyAsync(&v, dptr, sizeof(T), cudaMemcpyDeviceToHost, s));
  VASMG_CUDA(cudaStreamSynchronize(s));
  return v;
}

// ------------------------------------------------------------------ primitives (prims.cu)

// Exclusive prefix sum, in place allowed.  Returns nothing; total = out[n-1]+in[n-1].
void scan_exclusive_i64(const i64* in, i64* out, i64 n, cudaStream_t s);
void scan_exclusive_i32(const int32_t* in, int32_t* out, i64 n, cudaStream_t s);
// Stable LSD radix sort of u64 keys (low `bits` bits significant), optional
// int32 payload, in place.
void radix_sort(u64* keys, int32_t* vals, i64 n, int bits, cudaStream_t s);
// Compact sorted keys to their distinct values; returns the new count.
i64 unique_sorted(u64* keys, i64 n, cudaStream_t s);
// Row pointers of a sorted (row << 32 | col) key array: rp[r] = first key >= r<<32.
void rowptr_from_pairs(const u64* keys, i64 nnz, i64 nrows, int32_t* rp, cudaStream_t s);
// Min and max of a double array.
void minmax_f64(const double* x, i64 n, double* mn, double* mx, cudaStream_t s);
int32_t max_i32(const int32_t* x, i64 n, cudaStream_t s);
i64 sum_i64(const i64* x, i64 n, cudaStream_t s);

int bits_for(u64 maxval);

// ------------------------------------------------------------------ hierarchy

// A level in canonical order (level 0: input vertex ids; level >= 1: ascending
// lattice key).  Full BSR with the diagonal block, FP64, row-major d x d blocks.
struct CanonLevel {
  i64 nv = 0, nnzb = 0;
  DevBuf<int32_t> rp, ci;
  DevBuf<double> v;
  DevBuf<uint8_t> dead;         // nv*d
  DevBuf<u64> lat;              // level >= 1: lattice-corner keys
  i64 ncells = 0;
  DevBuf<u64> cell_start;       // level >= 1: cells sorted by start key (d*K bits)
  DevBuf<uint8_t> cell_depth;
  int max_depth = 0;
  // interpolation to the next coarser level (rows: this level)
  i64 pnnz = 0;
  DevBuf<int32_t> prp, pci;
  DevBuf<double> pw;
  // R = P^T as (coarse row, fine entry) pairs, kept for recomputing the
  // Galerkin values of the next level when the material changes
  DevBuf<u64> r_keys;
  DevBuf<int32_t> r_ent, r_rp;
  // colouring
  DevBuf<int32_t> colour;
  int ncol = 0;
  DevBuf<double> dinv;          // nv*d*d
};

// A level in solve order: vertices renumbered colour by colour (each colour a
// contiguous range), off-diagonal blocks only, values as separate planes
// (structure of arrays, plane q = block entry q of the d x d block).
struct SolveLevel {
  i64 nv = 0, nnz = 0;
  int ncol = 0;
  std::vector<int32_t> cs;      // host copy of colour starts [ncol+1]
  std::vector<uint32_t> sec;    // host: spatial key of each solve row (ascending within a colour)
  DevBuf<int32_t> ent;          // canonical block entry of each solve-order off-diagonal entry
  DevBuf<int32_t> perm, iperm;  // solve index -> canonical, canonical -> solve
  DevBuf<int32_t> rp, ci, sp;   // sp[i]: first entry of row i whose column is of a later colour
  DevBuf<double> off64;         // off-diagonal blocks, layout block_index()
  DevBuf<float> off32;
  DevBuf<__nv_bfloat16> off16;
  DevBuf<double> diag64;        // level 0: [d*d][nv]
  DevBuf<double> dinv64;        // [d*d][nv]
  DevBuf<float> dinv32;
  DevBuf<uint8_t> deadbits;     // per vertex, bit a set = component a removed
  // transfers to level l+1 (solve order on both sides)
  DevBuf<int32_t> prp, pci, rrp, rci;
  DevBuf<double> pw64, rw64;
  DevBuf<float> pw32, rw32;
  // V-cycle work vectors (precision of the V-cycle)
  DevBuf<char> x, b, r;
};

struct EngineBase;

struct Ctx {
  int dim = 2, K = 31, T = 4, precision = VASMG_FP64, max_iters = 1000, use_graph = 1;
  int max_ctas = 0;       // cap on the CTAs of one sweep launch (0: device capacity)
  int dense_coarse = 1;   // FP32-vector modes: apply the cycle below the dense level as one matrix
  int autotune = 1;       // measure the lanes per row of each region level at setup
  int gamma = 1;          // coarse corrections per level (1: V-cycle, 2: W-cycle)
  int additive = 0;       // preconditioner S + P B_1 P^T (Sec. 4) instead of the cycle from level 0
  int ctas_used = 0;      // largest sweep grid this handle launches
  int cta_capacity = 0;   // CTAs of the sweep kernels the device holds at once
  i64 coarse_max_dofs = 0;
  cudaStream_t stream = 0;       // internal non-blocking stream owned by the handle
  cudaStream_t user_stream = 0;  // caller's stream (options.stream)
  cudaEvent_t join_ev = nullptr;
  int device = -1;               // the device current at vasmg_setup; all of the handle's memory is there
  // recorded on the caller's stream after each vasmg_coarse_solve_noalloc
  // kernel; vasmg_update_data waits for it before refilling the factor
  cudaEvent_t noalloc_ev = nullptr;
  i64 nv = 0, ne = 0, n = 0;
  double setup_ms = 0;
  // inputs
  DevBuf<double> X, lam, mu, vol;
  DevBuf<int32_t> E;
  DevBuf<uint8_t> isdir;
  DevBuf<double> udir, lift;
  bool has_dir_values = false;
  std::vector<int64_t> dir_dofs;  // host: the Dirichlet dofs in the caller's order
  double update_ms = 0;           // wall-clock of the last vasmg_update_data
  // vertex -> element incidence
  DevBuf<int32_t> inc_rp, inc_e;
  // region tree
  double box_m = 0, box_M = 0;
  DevBuf<u64> mkey;             // per input vertex
  DevBuf<int32_t> morder;       // vertices sorted by Morton key
  DevBuf<uint8_t> leaf_depth;   // per input vertex
  DevBuf<u64> leaf_start;       // per input vertex (cell start key)
  std::vector<CanonLevel> C;
  std::vector<SolveLevel> S;
  // coarsest dense factor (FP64), in solve order of the last level
  i64 nc = 0;
  DevBuf<double> chol;
  DevBuf<uint8_t> chol_drop;
  // solve engine (solve.cu): kernels specialised for dim and precision
  struct EngineBase* eng = nullptr;
  i64 last_launches = 0;
  // scratch for vasmg_apply
  DevBuf<double> tmp_a, tmp_b;
};

// Order the handle's internal stream after all work already queued on the
// caller's stream.
inline void join_user(Ctx& c) {
  VASMG_CUDA(cudaEventRecord(c.join_ev, c.user_stream));
  VASMG_CUDA(cudaStreamWaitEvent(c.stream, c.join_ev, 0));
}

// setup stages
void setup_assemble(Ctx& c);                       // setup_assemble.cu
void assemble_load_dev(Ctx& c, const double* f, double* F_dev);
void setup_tree(Ctx& c);                           // setup_tree.cu
void setup_galerkin(Ctx& c, int l);                // setup_galerkin.cu
void setup_colour_and_solve_levels(Ctx& c);        // setup_colour.cu
// numeric stages only (the structure from setup stays): for new Lame
// parameters or Dirichlet values
void assemble_values(Ctx& c);                      // setup_assemble.cu
void galerkin_values(Ctx& c, int l);               // setup_galerkin.cu
void solve_level_values(Ctx& c);                   // setup_colour.cu
void refresh_solver_values(Ctx& c);                // solve.cu
void setup_solver_state(Ctx& c);                   // solve.cu
// solve
int solve_dev(Ctx& c, const double* F_dev, double* U_dev, double tol, vasmg_stats* st);
void apply_op(Ctx& c, int op, int level, const double* x_dev, double* y_dev);
double time_kernel(Ctx& c, int which, int level, int reps, double* bytes);
int solve_multi_dev(Ctx& c, int k, const double* const* F, double* const* U, double tol, vasmg_stats* st);
int solve_batch_dev(const std::vector<Ctx*>& cs, const double* const* F, double* const* U, double tol,
                    vasmg_stats* st, i64* launches);
double time_kernel_multi(Ctx& c, int which, int level, int k, int reps, double* bytes);
void dense_level_info(Ctx& c, int* kd, int* dn);  // the engine's dense level, (-1, 0) if none
void lanes_info(Ctx& c, int32_t* g, int n);       // lanes per row of the region levels, 0 elsewhere
void staged_info(Ctx& c, int level, int64_t* v);  // a level's staged sweep copies (see VASMG_EXPORT_STAGED)
int probe_wait_timeout(double* elapsed_ms);       // the bounded device wait run out on purpose
int probe_fp64_rate(double* tflops, double* ms);  // FP64 FMA throughput of the current device
void destroy_solver_state(Ctx& c);

// small device helpers shared across files
__host__ __device__ inline u64 part1by1(u64 x) {
  x &= 0x00000000FFFFFFFFull;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}
__host__ __device__ inline u64 compact1by1(u64 x) {
  x &= 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
  x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
  x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
  return x;
}
__host__ __device__ inline u64 part1by2(u64 x) {
  x &= 0x1FFFFFull;  // 21 bits
  x = (x | (x << 32)) & 0x1F00000000FFFFull;
  x = (x | (x << 16)) & 0x1F0000FF0000FFull;
  x = (x | (x << 8)) & 0x100F00F00F00F00Full;
  x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}
__host__ __device__ inline u64 compact1by2(u64 x) {
  x &= 0x1249249249249249ull;
  x = (x | (x >> 2)) & 0x10C30C30C30C30C3ull;
  x = (x | (x >> 4)) & 0x100F00F00F00F00Full;
  x = (x | (x >> 8)) & 0x1F0000FF0000FFull;
  x = (x | (x >> 16)) & 0x1F00000000FFFFull;
  x = (x | (x >> 32)) & 0x1FFFFFull;
  return x;
}
// Morton interleave of d coordinates (bit b of axis a -> bit b*d + a).
__host__ __device__ inline u64 morton(const u64* c, int d) {
  return d == 2 ? (part1by1(c[0]) | (part1by1(c[1]) << 1))
                : (part1by2(c[0]) | (part1by2(c[1]) << 1) | (part1by2(c[2]) << 2));
}
__host__ __device__ inline void unmorton(u64 k, int d, u64* c) {
  if (d == 2) {
    c[0] = compact1by1(k);
    c[1] = compact1by1(k >> 1);
  } else {
    c[0] = compact1by2(k);
    c[1] = compact1by2(k >> 1);
    c[2] = compact1by2(k >> 2);
  }
}

// splitmix64 output function (Steele, Lea, Flood 2014; Vigna's constants):
// the colouring priority of vertex v is splitmix64(v).
__host__ __device__ inline u64 splitmix64(u64 x) {
  u64 z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Storage of component q (row-major in the d x d block) of block k among n
// blocks: 2 x 2 blocks are stored contiguously (one 8- or 16-byte load per
// block); of a 3 x 3 block the first 8 components are stored contiguously
// (one 16-byte load in BF16, two in FP32, four in FP64) and the ninth in a
// plane of n values after them, so a block costs 2, 3 or 5 loads instead of
// 9 and no padding.
__host__ __device__ inline long long block_index(int q, long long k, long long n, int dd) {
  if (dd == 4) return k * 4 + q;
  if (dd == 9) return q < 8 ? k * 8 + q : 8 * n + k;
  return (long long)q * n + k;
}

// Forward and backward substitution with a dense lower Cholesky factor L
// (row-major n x n, FP64) by one warp, in place on y[0..n): y <- L^{-T} L^{-1} y.
// A dropped pivot (drop[j] != 0) removes direction j: y_j is set to 0 in both
// passes.  Used by the coarsest-level solves of the V-cycle and of
// vasmg_coarse_solve_noalloc.
__device__ __forceinline__ void chol_substitute_warp(const double* chol, const uint8_t* drop, int n, double* y) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < n; ++j) {
    const double ljj = chol[(long long)j * n + j];
    const double yj = drop[j] ? 0.0 : y[j] / ljj;
    __syncwarp();
    if (lane == 0) y[j] = yj;
    for (int i = j + 1 + lane; i < n; i += 32) y[i] -= chol[(long long)i * n + j] * yj;
    __syncwarp();
  }
  for (int j = n - 1; j >= 0; --j) {
    const double ljj = chol[(long long)j * n + j];
    const double xj = drop[j] ? 0.0 : y[j] / ljj;
    __syncwarp();
    if (lane == 0) y[j] = xj;
    for (int i = lane; i < j; i += 32) y[i] -= chol[(long long)j * n + i] * xj;
    __syncwarp();
  }
}

inline int grid_for(i64 n, int threads, int cap = 1 << 20) {
  i64 g = ceil_div(n, threads);
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace vasmg
