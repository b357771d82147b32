// Galerkin coarse operators A_{l+1} = P^T A_l P (eq. (R), eq. (Ac)) on the
// device, with P = P_s (x) I_d and the rows of dead fine dofs masked.
//
// Pattern: the structural block product of P_s^T pattern(A_l) P_s plus the
// diagonal (pairs (I, J) generated per fine vertex, each fine vertex's coarse
// columns made unique locally first, then radix sorted and made unique).
// Values: one warp per coarse row I sums, in ascending fine index i and then
// ascending block k of row i, w_iI (M A_l M)_ij w_jJ into its row -- a fixed
// order, so the result is deterministic.  Coarse dofs whose masked column of
// P is empty are dead and get identity rows.
#include "common.cuh"

namespace vasmg {

// Coarse columns a fine row i reaches: the union over the blocks k of A_l's
// row i of the columns of P's row j_k.  Up to GAL_UNION of them are collected,
// sorted and made unique in thread-local storage, so that each (I, J) pair is
// emitted once per fine row; a row with a longer candidate list emits its
// list as it is (the global sort and unique below remove the repeats either
// way, so the pattern is the same).
constexpr int GAL_UNION = 128;

__device__ __forceinline__ int gal_row_union(const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                             const int32_t* __restrict__ prp, const int32_t* __restrict__ pci,
                                             i64 i, int32_t* cols) {
  int n = 0;
  for (int32_t k = arp[i]; k < arp[i + 1]; ++k) {
    const int32_t j = aci[k];
    for (int32_t b = prp[j]; b < prp[j + 1]; ++b) {
      if (n == GAL_UNION) return -1;
      // insertion into the sorted prefix, skipping a repeat
      const int32_t J = pci[b];
      int p = n;
      while (p > 0 && cols[p - 1] > J) --p;
      if (p > 0 && cols[p - 1] == J) continue;
      for (int q = n; q > p; --q) cols[q] = cols[q - 1];
      cols[p] = J;
      ++n;
    }
  }
  return n;
}

__global__ void gal_count_kernel(const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                 const int32_t* __restrict__ prp, const int32_t* __restrict__ pci, i64 nf,
                                 long long* __restrict__ cnt) {
  int32_t cols[GAL_UNION];
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (i64)gridDim.x * blockDim.x) {
    long long s = gal_row_union(arp, aci, prp, pci, i, cols);
    if (s < 0) {
      s = 0;
      for (int32_t k = arp[i]; k < arp[i + 1]; ++k) {
        const int32_t j = aci[k];
        s += prp[j + 1] - prp[j];
      }
    }
    cnt[i] = s * (long long)(prp[i + 1] - prp[i]);
  }
}

__global__ void gal_pairs_kernel(const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                 const int32_t* __restrict__ prp, const int32_t* __restrict__ pci, i64 nf,
                                 const long long* __restrict__ off, u64* __restrict__ keys) {
  int32_t cols[GAL_UNION];
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (i64)gridDim.x * blockDim.x) {
    long long o = off[i];
    const int nu = gal_row_union(arp, aci, prp, pci, i, cols);
    for (int32_t a = prp[i]; a < prp[i + 1]; ++a) {
      const u64 I = (uint32_t)pci[a];
      if (nu >= 0) {
        for (int q = 0; q < nu; ++q) keys[o++] = (I << 32) | (uint32_t)cols[q];
      } else {
        for (int32_t k = arp[i]; k < arp[i + 1]; ++k) {
          const int32_t j = aci[k];
          for (int32_t b = prp[j]; b < prp[j + 1]; ++b) keys[o++] = (I << 32) | (uint32_t)pci[b];
        }
      }
    }
  }
}

__global__ void diag_pairs_kernel(i64 nc, u64* __restrict__ keys) {
  for (i64 I = (i64)blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += (i64)gridDim.x * blockDim.x)
    keys[I] = ((u64)I << 32) | (u64)I;
}

__global__ void transpose_keys_kernel(const int32_t* __restrict__ prp, const int32_t* __restrict__ pci, i64 nf,
                                      u64* __restrict__ keys, int32_t* __restrict__ vals) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (i64)gridDim.x * blockDim.x)
    for (int32_t a = prp[i]; a < prp[i + 1]; ++a) {
      keys[a] = ((u64)(uint32_t)pci[a] << 32) | (u64)i;
      vals[a] = a;
    }
}

__global__ void low32_i_kernel(const u64* __restrict__ k, i64 n, int32_t* __restrict__ out) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    out[i] = (int32_t)(k[i] & 0xffffffffull);
}

// One warp per coarse row I.  The warp walks the items (t, k) of the row -- an
// R entry t (fine vertex i, weight w_iI) and a block k of A_l's row i (column
// j) -- in ascending t, then ascending k; the lanes split the (b, r, s) terms
// of one item (b over the entries of P_j's row, (r, s) over the block), and
// those all land on different scalars of row I, since the columns of one
// row of P are distinct.  Every scalar thus receives its terms in the same
// order as a single thread walking the row would add them.  The warp's
// lanes then write the dead masks and identity rows.
template <int D>
__global__ void gal_values_kernel(
    i64 nc, const int32_t* __restrict__ rrp, const int32_t* __restrict__ rent, const u64* __restrict__ rkeys,
    const int32_t* __restrict__ prp, const int32_t* __restrict__ pci, const double* __restrict__ pw,
    const int32_t* __restrict__ arp, const int32_t* __restrict__ aci, const double* __restrict__ av,
    const uint8_t* __restrict__ fdead, const int32_t* __restrict__ crp, const int32_t* __restrict__ cci,
    double* __restrict__ cv, uint8_t* __restrict__ cdead) {
  constexpr int DD = D * D;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const i64 nwarps = (i64)gridDim.x * (blockDim.x >> 5);
  for (i64 I = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; I < nc; I += nwarps) {
    const int32_t c0 = crp[I], c1 = crp[I + 1];
    unsigned alive = 0;
    for (int32_t t = rrp[I]; t < rrp[I + 1]; ++t) {
      const i64 i = (i64)(rkeys[t] & 0xffffffffull);
      const double wI = pw[rent[t]];
      unsigned fi = 0;
#pragma unroll
      for (int r = 0; r < D; ++r) fi |= fdead[i * D + r] ? 0u : 1u << r;
      alive |= fi;
      const int32_t k0 = arp[i], k1 = arp[i + 1];
      for (int32_t kb = k0; kb < k1; kb += 32) {
        const int nk = min(32, k1 - kb);
        // the lanes fetch the column data of up to 32 items at once
        int32_t p0l = 0, p1l = 0;
        unsigned fjl = 0;
        if (lane < nk) {
          const i64 j = aci[kb + lane];
          p0l = prp[j];
          p1l = prp[j + 1];
#pragma unroll
          for (int s = 0; s < D; ++s) fjl |= fdead[j * D + s] ? 0u : 1u << s;
        }
        for (int q = 0; q < nk; ++q) {
          const int32_t p0 = __shfl_sync(FULL, p0l, q), p1 = __shfl_sync(FULL, p1l, q);
          const unsigned fj = __shfl_sync(FULL, fjl, q);
          const double* B = av + (i64)(kb + q) * DD;
          const int nterm = (p1 - p0) * DD;
          for (int e = lane; e < nterm; e += 32) {
            const int bq = e / DD, rs = e - bq * DD, r = rs / D, sc = rs - r * D;
            if (!((fi >> r) & 1u) || !((fj >> sc) & 1u)) continue;
            const int32_t J = pci[p0 + bq];
            const double wJ = pw[p0 + bq];
            int32_t lo = c0, hi = c1;
            while (lo < hi) {
              const int32_t mid = (lo + hi) >> 1;
              if (cci[mid] < J) lo = mid + 1; else hi = mid;
            }
            double* C = cv + (i64)lo * DD + rs;
            *C = __dadd_rn(*C, __dmul_rn(__dmul_rn(wI, B[rs]), wJ));
          }
          // the next item may add to a scalar another lane just wrote
          __syncwarp();
        }
      }
    }
    // dead coarse dofs -> identity rows (their masked column of P is empty)
    if (lane < D) {
      int32_t lo = c0, hi = c1;
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (cci[mid] < (int32_t)I) lo = mid + 1; else hi = mid;
      }
      const bool al = (alive >> lane) & 1u;
      cdead[I * D + lane] = al ? 0 : 1;
      if (!al) cv[(i64)lo * DD + lane * D + lane] = 1.0;
    }
    __syncwarp();
  }
}

void setup_galerkin(Ctx& c, int l) {
  cudaStream_t s = c.stream;
  const int d = c.dim;
  CanonLevel& f = c.C[l];
  CanonLevel& g = c.C[l + 1];
  // ---- symbolic
  DevBuf<long long> cnt;
  cnt.alloc(f.nv + 1, s);
  cnt.zero();
  gal_count_kernel<<<grid_for(f.nv, 256), 256, 0, s>>>(f.rp.get(), f.ci.get(), f.prp.get(), f.pci.get(), f.nv,
                                                        cnt.get());
  check_launch("gal_count");
  scan_exclusive_i64((const i64*)cnt.get(), (i64*)cnt.get(), f.nv + 1, s);
  const i64 m = fetch(cnt.get() + f.nv, s);
  DevBuf<u64> keys;
  keys.alloc(m + g.nv, s);
  gal_pairs_kernel<<<grid_for(f.nv, 128), 128, 0, s>>>(f.rp.get(), f.ci.get(), f.prp.get(), f.pci.get(), f.nv,
                                                        cnt.get(), keys.get());
  check_launch("gal_pairs");
  diag_pairs_kernel<<<grid_for(g.nv, 256), 256, 0, s>>>(g.nv, keys.get() + m);
  check_launch("diag_pairs");
  radix_sort(keys.get(), nullptr, m + g.nv, 32 + bits_for((u64)g.nv), s);
  g.nnzb = unique_sorted(keys.get(), m + g.nv, s);
  VASMG_CHECK(g.nnzb < (i64)INT32_MAX, VASMG_ERR_UNSUPPORTED, "too many blocks for 32-bit indices");
  g.rp.alloc(g.nv + 1, s);
  g.ci.alloc(g.nnzb, s);
  rowptr_from_pairs(keys.get(), g.nnzb, g.nv, g.rp.get(), s);
  low32_i_kernel<<<grid_for(g.nnzb, 256), 256, 0, s>>>(keys.get(), g.nnzb, g.ci.get());
  check_launch("low32");
  keys.release();
  // ---- R = P^T as (coarse row, fine index) sorted pairs, kept on the fine level
  f.r_keys.alloc(f.pnnz, s);
  f.r_ent.alloc(f.pnnz, s);
  transpose_keys_kernel<<<grid_for(f.nv, 256), 256, 0, s>>>(f.prp.get(), f.pci.get(), f.nv, f.r_keys.get(),
                                                             f.r_ent.get());
  check_launch("transpose_keys");
  radix_sort(f.r_keys.get(), f.r_ent.get(), f.pnnz, 32 + bits_for((u64)g.nv), s);
  f.r_rp.alloc(g.nv + 1, s);
  rowptr_from_pairs(f.r_keys.get(), f.pnnz, g.nv, f.r_rp.get(), s);
  galerkin_values(c, l);
}

// ---- numeric: A_{l+1} = P^T A_l P on the pattern built above (eq. (Ac)),
// with dead-dof masks; also run again when A_l's values change.
void galerkin_values(Ctx& c, int l) {
  cudaStream_t s = c.stream;
  const int d = c.dim;
  CanonLevel& f = c.C[l];
  CanonLevel& g = c.C[l + 1];
  if (g.v.n != g.nnzb * d * d) g.v.alloc(g.nnzb * d * d, s);
  g.v.zero();
  if (g.dead.n != g.nv * d) g.dead.alloc(g.nv * d, s);
  if (d == 2)
    gal_values_kernel<2><<<grid_for(g.nv * 32, 256), 256, 0, s>>>(g.nv, f.r_rp.get(), f.r_ent.get(), f.r_keys.get(),
                                                              f.prp.get(), f.pci.get(), f.pw.get(), f.rp.get(),
                                                              f.ci.get(), f.v.get(), f.dead.get(), g.rp.get(),
                                                              g.ci.get(), g.v.get(), g.dead.get());
  else
    gal_values_kernel<3><<<grid_for(g.nv * 32, 256), 256, 0, s>>>(g.nv, f.r_rp.get(), f.r_ent.get(), f.r_keys.get(),
                                                              f.prp.get(), f.pci.get(), f.pw.get(), f.rp.get(),
                                                              f.ci.get(), f.v.get(), f.dead.get(), g.rp.get(),
                                                              g.ci.get(), g.v.get(), g.dead.get());
  check_launch("gal_values");
}

}  // namespace vasmg
