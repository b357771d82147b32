// Galerkin coarse operators A_{l+1} = P^T A_l P (eq. (R), eq. (Ac)) on the
// device, with P = P_s (x) I_d and the rows of dead fine dofs masked.
//
// Pattern: the structural block product of P_s^T pattern(A_l) P_s plus the
// diagonal (pairs (I, J) generated per fine vertex, radix sorted, made unique).
// Values: one thread per coarse row I sums, in ascending fine index i and then
// ascending block k of row i, w_iI (M A_l M)_ij w_jJ into its row -- a fixed
// order, so the result is deterministic.  Coarse dofs whose masked column of
// P is empty are dead and get identity rows.
#include "common.cuh"

namespace vasmg {

__global__ void gal_count_kernel(const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                 const int32_t* __restrict__ prp, i64 nf, long long* __restrict__ cnt) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (i64)gridDim.x * blockDim.x) {
    long long s = 0;
    for (int32_t k = arp[i]; k < arp[i + 1]; ++k) {
      const int32_t j = aci[k];
      s += prp[j + 1] - prp[j];
    }
    cnt[i] = s * (long long)(prp[i + 1] - prp[i]);
  }
}

__global__ void gal_pairs_kernel(const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                 const int32_t* __restrict__ prp, const int32_t* __restrict__ pci, i64 nf,
                                 const long long* __restrict__ off, u64* __restrict__ keys) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (i64)gridDim.x * blockDim.x) {
    long long o = off[i];
    for (int32_t a = prp[i]; a < prp[i + 1]; ++a) {
      const u64 I = (uint32_t)pci[a];
      for (int32_t k = arp[i]; k < arp[i + 1]; ++k) {
        const int32_t j = aci[k];
        for (int32_t b = prp[j]; b < prp[j + 1]; ++b) keys[o++] = (I << 32) | (uint32_t)pci[b];
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

template <int D>
__global__ void gal_values_kernel(i64 nc, const int32_t* __restrict__ rrp, const int32_t* __restrict__ rent,
                                  const u64* __restrict__ rkeys, const int32_t* __restrict__ prp,
                                  const int32_t* __restrict__ pci, const double* __restrict__ pw,
                                  const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                  const double* __restrict__ av, const uint8_t* __restrict__ fdead,
                                  const int32_t* __restrict__ crp, const int32_t* __restrict__ cci,
                                  double* __restrict__ cv, uint8_t* __restrict__ cdead) {
  constexpr int DD = D * D;
  for (i64 I = (i64)blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += (i64)gridDim.x * blockDim.x) {
    const int32_t c0 = crp[I], c1 = crp[I + 1];
    bool alive[D];
#pragma unroll
    for (int r = 0; r < D; ++r) alive[r] = false;
    for (int32_t t = rrp[I]; t < rrp[I + 1]; ++t) {
      const i64 i = (i64)(rkeys[t] & 0xffffffffull);
      const double wI = pw[rent[t]];
      bool fi[D];
#pragma unroll
      for (int r = 0; r < D; ++r) {
        fi[r] = !fdead[i * D + r];
        alive[r] = alive[r] || fi[r];
      }
      for (int32_t k = arp[i]; k < arp[i + 1]; ++k) {
        const i64 j = aci[k];
        const double* B = av + (i64)k * DD;
        bool fj[D];
#pragma unroll
        for (int s = 0; s < D; ++s) fj[s] = !fdead[j * D + s];
        for (int32_t b = prp[j]; b < prp[j + 1]; ++b) {
          const int32_t J = pci[b];
          const double wJ = pw[b];
          int32_t lo = c0, hi = c1;
          while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (cci[mid] < J) lo = mid + 1; else hi = mid;
          }
          double* C = cv + (i64)lo * DD;
#pragma unroll
          for (int r = 0; r < D; ++r) {
            if (!fi[r]) continue;
#pragma unroll
            for (int s = 0; s < D; ++s) {
              if (!fj[s]) continue;
              C[r * D + s] = __dadd_rn(C[r * D + s], __dmul_rn(__dmul_rn(wI, B[r * D + s]), wJ));
            }
          }
        }
      }
    }
    // dead coarse dofs -> identity rows (their masked column of P is empty)
    int32_t lo = c0, hi = c1;
    while (lo < hi) {
      const int32_t mid = (lo + hi) >> 1;
      if (cci[mid] < (int32_t)I) lo = mid + 1; else hi = mid;
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
      cdead[I * D + r] = alive[r] ? 0 : 1;
      if (!alive[r]) cv[(i64)lo * DD + r * D + r] = 1.0;
    }
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
  gal_count_kernel<<<grid_for(f.nv, 256), 256, 0, s>>>(f.rp.get(), f.ci.get(), f.prp.get(), f.nv, cnt.get());
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
    gal_values_kernel<2><<<grid_for(g.nv, 128), 128, 0, s>>>(g.nv, f.r_rp.get(), f.r_ent.get(), f.r_keys.get(),
                                                              f.prp.get(), f.pci.get(), f.pw.get(), f.rp.get(),
                                                              f.ci.get(), f.v.get(), f.dead.get(), g.rp.get(),
                                                              g.ci.get(), g.v.get(), g.dead.get());
  else
    gal_values_kernel<3><<<grid_for(g.nv, 128), 128, 0, s>>>(g.nv, f.r_rp.get(), f.r_ent.get(), f.r_keys.get(),
                                                              f.prp.get(), f.pci.get(), f.pw.get(), f.rp.get(),
                                                              f.ci.get(), f.v.get(), f.dead.get(), g.rp.get(),
                                                              g.ci.get(), g.v.get(), g.dead.get());
  check_launch("gal_values");
}

}  // namespace vasmg
