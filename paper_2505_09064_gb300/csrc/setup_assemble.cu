// Device assembly of the P1 elasticity stiffness matrix and load vector
// (Sec. 2: the block form of A with A_11 = int Phi_x^T Phi_x etc., written for
// d = 2, 3 as K_ij[a][b] = |K| (lam g_ia g_jb + mu g_ib g_ja + mu delta_ab
// g_i . g_j)), and the Dirichlet rows.
//
// Determinism: every row is owned by one thread, which adds the element
// contributions of that row in ascending element order.  Block (j,i) is then
// formed from exactly the same products, in the same order, as the transpose
// of block (i,j), so A is bitwise symmetric.
#include "common.cuh"

namespace vasmg {

__global__ void check_elements_kernel(const int32_t* __restrict__ E, i64 nentries, i64 nv, int* __restrict__ bad) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nentries; i += (i64)gridDim.x * blockDim.x)
    if (E[i] < 0 || E[i] >= nv) atomicOr(bad, 1);
}

__global__ void incidence_keys_kernel(const int32_t* __restrict__ E, i64 ne, int nl, u64* __restrict__ keys,
                                      int32_t* __restrict__ vals) {
  const i64 m = ne * nl;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (i64)gridDim.x * blockDim.x) {
    keys[i] = (u64)(uint32_t)E[i];
    vals[i] = (int32_t)(i / nl);
  }
}

__global__ void rowptr_plain_kernel(const u64* __restrict__ keys, i64 m, i64 nrows, int32_t* __restrict__ rp) {
  for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r <= nrows; r += (i64)gridDim.x * blockDim.x) {
    i64 lo = 0, hi = m;
    while (lo < hi) {
      i64 mid = (lo + hi) >> 1;
      if (keys[mid] < (u64)r) lo = mid + 1; else hi = mid;
    }
    rp[r] = (int32_t)lo;
  }
}

__global__ void pattern_pairs_kernel(const int32_t* __restrict__ E, i64 ne, int nl, i64 nv, u64* __restrict__ keys) {
  const i64 per = (i64)nl * nl;
  const i64 m = ne * per;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < m + nv; i += (i64)gridDim.x * blockDim.x) {
    if (i < m) {
      const i64 e = i / per;
      const int rc = (int)(i - e * per);
      const u64 a = (uint32_t)E[e * nl + rc / nl], b = (uint32_t)E[e * nl + rc % nl];
      keys[i] = (a << 32) | b;
    } else {
      const u64 v = (u64)(i - m);
      keys[i] = (v << 32) | v;
    }
  }
}

__global__ void low32_kernel(const u64* __restrict__ k, i64 n, int32_t* __restrict__ out) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    out[i] = (int32_t)(k[i] & 0xffffffffull);
}

// Barycentric gradients of the P1 basis and the measure of simplex e.
template <int D>
__device__ bool p1_grad(const double* __restrict__ X, const int32_t* __restrict__ v, double g[D + 1][D],
                        double* meas) {
  double J[D][D];
#pragma unroll
  for (int k = 0; k < D; ++k)
#pragma unroll
    for (int a = 0; a < D; ++a) J[a][k] = __dsub_rn(X[(i64)v[k + 1] * D + a], X[(i64)v[0] * D + a]);
  if (D == 2) {
    const double det = __dsub_rn(__dmul_rn(J[0][0], J[1][1]), __dmul_rn(J[0][1], J[1][0]));
    if (!(det != 0.0) || !isfinite(det)) return false;
    g[1][0] = J[1][1] / det;
    g[1][1] = -J[0][1] / det;
    g[2][0] = -J[1][0] / det;
    g[2][1] = J[0][0] / det;
    *meas = fabs(det) * 0.5;
  } else {
    // adjugate: inv = adj(J) / det; gradient of basis k+1 = row k of inv
    double c[3][3];
    c[0][0] = __dsub_rn(__dmul_rn(J[1][1], J[2][2]), __dmul_rn(J[1][2], J[2][1]));
    c[1][0] = __dsub_rn(__dmul_rn(J[1][2], J[2][0]), __dmul_rn(J[1][0], J[2][2]));
    c[2][0] = __dsub_rn(__dmul_rn(J[1][0], J[2][1]), __dmul_rn(J[1][1], J[2][0]));
    c[0][1] = __dsub_rn(__dmul_rn(J[0][2], J[2][1]), __dmul_rn(J[0][1], J[2][2]));
    c[1][1] = __dsub_rn(__dmul_rn(J[0][0], J[2][2]), __dmul_rn(J[0][2], J[2][0]));
    c[2][1] = __dsub_rn(__dmul_rn(J[0][1], J[2][0]), __dmul_rn(J[0][0], J[2][1]));
    c[0][2] = __dsub_rn(__dmul_rn(J[0][1], J[1][2]), __dmul_rn(J[0][2], J[1][1]));
    c[1][2] = __dsub_rn(__dmul_rn(J[0][2], J[1][0]), __dmul_rn(J[0][0], J[1][2]));
    c[2][2] = __dsub_rn(__dmul_rn(J[0][0], J[1][1]), __dmul_rn(J[0][1], J[1][0]));
    const double det =
        __dadd_rn(__dadd_rn(__dmul_rn(J[0][0], c[0][0]), __dmul_rn(J[0][1], c[1][0])), __dmul_rn(J[0][2], c[2][0]));
    if (!(det != 0.0) || !isfinite(det)) return false;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int a = 0; a < 3; ++a) g[k + 1][a] = c[k][a] / det;
    *meas = fabs(det) / 6.0;
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double s = g[1][a];
#pragma unroll
    for (int k = 2; k <= D; ++k) s = __dadd_rn(s, g[k][a]);
    g[0][a] = -s;
  }
  return true;
}

template <int D>
__global__ void assemble_values_kernel(const double* __restrict__ X, const int32_t* __restrict__ E,
                                       const double* __restrict__ lam, const double* __restrict__ mu,
                                       const int32_t* __restrict__ inc_rp, const int32_t* __restrict__ inc_e,
                                       const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                       double* __restrict__ val, double* __restrict__ vol, i64 nv,
                                       int* __restrict__ bad) {
  constexpr int NL = D + 1, DD = D * D;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (i64)gridDim.x * blockDim.x) {
    const int32_t r0 = rp[i], r1 = rp[i + 1];
    for (int32_t t = inc_rp[i]; t < inc_rp[i + 1]; ++t) {
      const int32_t e = inc_e[t];
      const int32_t* v = E + (i64)e * NL;
      double g[NL][D], meas;
      if (!p1_grad<D>(X, v, g, &meas)) {
        atomicOr(bad, 2);
        continue;
      }
      int r = 0;
      while (v[r] != (int32_t)i) ++r;
      if (r == 0) vol[e] = meas;
      const double la = lam[e], m = mu[e];
#pragma unroll
      for (int c = 0; c < NL; ++c) {
        // column position of vertex v[c] in row i
        int32_t lo = r0, hi = r1;
        while (lo < hi) {
          int32_t mid = (lo + hi) >> 1;
          if (ci[mid] < v[c]) lo = mid + 1; else hi = mid;
        }
        double* B = val + (i64)lo * DD;
        double gg = __dmul_rn(g[r][0], g[c][0]);
#pragma unroll
        for (int x = 1; x < D; ++x) gg = __dadd_rn(gg, __dmul_rn(g[r][x], g[c][x]));
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) {
            double t1 = __dmul_rn(la, __dmul_rn(g[r][a], g[c][b]));
            double t2 = __dmul_rn(m, __dmul_rn(g[r][b], g[c][a]));
            double s = __dadd_rn(t1, t2);
            if (a == b) s = __dadd_rn(s, __dmul_rn(m, gg));
            B[a * D + b] = __dadd_rn(B[a * D + b], __dmul_rn(meas, s));
          }
      }
    }
  }
}

// y = A x for the canonical full BSR (row-major blocks), FP64.
__global__ void canon_spmv_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                  const double* __restrict__ v, const double* __restrict__ x, double* __restrict__ y,
                                  i64 nv, int d) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (i64)gridDim.x * blockDim.x) {
    double acc[3] = {0, 0, 0};
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const i64 j = ci[k];
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) acc[a] += v[(i64)k * d * d + a * d + b] * x[j * d + b];
    }
    for (int a = 0; a < d; ++a) y[i * d + a] = acc[a];
  }
}

__global__ void dirichlet_rows_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                      double* __restrict__ v, const uint8_t* __restrict__ isdir, i64 nv, int d) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (i64)gridDim.x * blockDim.x) {
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const i64 j = ci[k];
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b)
          if (isdir[i * d + a] || isdir[j * d + b]) v[(i64)k * d * d + a * d + b] = (i == j && a == b) ? 1.0 : 0.0;
    }
  }
}

template <int D>
__global__ void load_kernel(const int32_t* __restrict__ inc_rp, const int32_t* __restrict__ inc_e,
                            const double* __restrict__ vol, double f0, double f1, double f2, double* __restrict__ F,
                            i64 nv) {
  const double f[3] = {f0, f1, f2};
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (i64)gridDim.x * blockDim.x) {
    double acc[D];
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] = 0.0;
    for (int32_t t = inc_rp[i]; t < inc_rp[i + 1]; ++t) {
      const double w = vol[inc_e[t]];
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] = __dadd_rn(acc[a], __dmul_rn(f[a], w) / (double)(D + 1));
    }
#pragma unroll
    for (int a = 0; a < D; ++a) F[i * D + a] = acc[a];
  }
}

void setup_assemble(Ctx& c) {
  cudaStream_t s = c.stream;
  const int d = c.dim, nl = d + 1;
  DevBuf<int> bad;
  bad.alloc(1, s);
  bad.zero();
  check_elements_kernel<<<grid_for(c.ne * nl, 256, 4096), 256, 0, s>>>(c.E.get(), c.ne * nl, c.nv, bad.get());
  check_launch("check_elements");
  VASMG_CHECK(fetch(bad.get(), s) == 0, VASMG_ERR_INVALID_ARG, "element vertex id out of range");

  // vertex -> element incidence (stable sort keeps elements ascending per vertex)
  {
    const i64 m = c.ne * nl;
    DevBuf<u64> keys;
    keys.alloc(m, s);
    c.inc_e.alloc(m, s);
    incidence_keys_kernel<<<grid_for(m, 256), 256, 0, s>>>(c.E.get(), c.ne, nl, keys.get(), c.inc_e.get());
    check_launch("incidence_keys");
    radix_sort(keys.get(), c.inc_e.get(), m, bits_for((u64)c.nv), s);
    c.inc_rp.alloc(c.nv + 1, s);
    rowptr_plain_kernel<<<grid_for(c.nv + 1, 256), 256, 0, s>>>(keys.get(), m, c.nv, c.inc_rp.get());
    check_launch("incidence_rowptr");
  }
  // block pattern: all vertex pairs sharing an element, plus the diagonal
  CanonLevel& L0 = c.C[0];
  L0.nv = c.nv;
  {
    const i64 m = c.ne * nl * nl + c.nv;
    DevBuf<u64> keys;
    keys.alloc(m, s);
    pattern_pairs_kernel<<<grid_for(m, 256), 256, 0, s>>>(c.E.get(), c.ne, nl, c.nv, keys.get());
    check_launch("pattern_pairs");
    radix_sort(keys.get(), nullptr, m, 32 + bits_for((u64)c.nv), s);
    const i64 nnz = unique_sorted(keys.get(), m, s);
    VASMG_CHECK(nnz < (i64)INT32_MAX, VASMG_ERR_UNSUPPORTED, "too many blocks for 32-bit indices");
    L0.nnzb = nnz;
    L0.rp.alloc(c.nv + 1, s);
    L0.ci.alloc(nnz, s);
    rowptr_from_pairs(keys.get(), nnz, c.nv, L0.rp.get(), s);
    low32_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(keys.get(), nnz, L0.ci.get());
    check_launch("low32");
  }
  assemble_values(c);
}

// Block values of A (Sec. 2) on the pattern built above, the Dirichlet lift
// A u_D and the identity rows/columns of the Dirichlet dofs.
void assemble_values(Ctx& c) {
  cudaStream_t s = c.stream;
  const int d = c.dim;
  CanonLevel& L0 = c.C[0];
  DevBuf<int> bad;
  bad.alloc(1, s);
  bad.zero();
  if (L0.v.n != L0.nnzb * d * d) L0.v.alloc(L0.nnzb * d * d, s);
  L0.v.zero();
  if (c.vol.n != c.ne) c.vol.alloc(c.ne, s);
  if (d == 2)
    assemble_values_kernel<2><<<grid_for(c.nv, 128), 128, 0, s>>>(c.X.get(), c.E.get(), c.lam.get(), c.mu.get(),
                                                                     c.inc_rp.get(), c.inc_e.get(), L0.rp.get(),
                                                                     L0.ci.get(), L0.v.get(), c.vol.get(), c.nv,
                                                                     bad.get());
  else
    assemble_values_kernel<3><<<grid_for(c.nv, 128), 128, 0, s>>>(c.X.get(), c.E.get(), c.lam.get(), c.mu.get(),
                                                                     c.inc_rp.get(), c.inc_e.get(), L0.rp.get(),
                                                                     L0.ci.get(), L0.v.get(), c.vol.get(), c.nv,
                                                                     bad.get());
  check_launch("assemble_values");
  VASMG_CHECK(fetch(bad.get(), s) == 0, VASMG_ERR_DEGENERATE_ELEMENT, "element with zero or non-finite measure");

  // Dirichlet: keep A u_D for the reduced right-hand side, then identity rows/columns
  if (c.lift.n != c.n) c.lift.alloc(c.n, s);
  canon_spmv_kernel<<<grid_for(c.nv, 128), 128, 0, s>>>(L0.rp.get(), L0.ci.get(), L0.v.get(), c.udir.get(),
                                                         c.lift.get(), c.nv, d);
  check_launch("lift");
  dirichlet_rows_kernel<<<grid_for(c.nv, 128), 128, 0, s>>>(L0.rp.get(), L0.ci.get(), L0.v.get(), c.isdir.get(),
                                                             c.nv, d);
  check_launch("dirichlet_rows");
  if (L0.dead.n != c.n) L0.dead.alloc(c.n, s);
  VASMG_CUDA(cudaMemcpyAsync(L0.dead.get(), c.isdir.get(), c.n, cudaMemcpyDeviceToDevice, s));
}

void assemble_load_dev(Ctx& c, const double* f, double* F_dev) {
  const double f0 = f[0], f1 = f[1], f2 = c.dim == 3 ? f[2] : 0.0;
  if (c.dim == 2)
    load_kernel<2><<<grid_for(c.nv, 256), 256, 0, c.stream>>>(c.inc_rp.get(), c.inc_e.get(), c.vol.get(), f0, f1, f2,
                                                               F_dev, c.nv);
  else
    load_kernel<3><<<grid_for(c.nv, 256), 256, 0, c.stream>>>(c.inc_rp.get(), c.inc_e.get(), c.vol.get(), f0, f1, f2,
                                                               F_dev, c.nv);
  check_launch("load");
}

}  // namespace vasmg
