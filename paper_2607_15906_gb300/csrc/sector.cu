// The method's steps on sector-layout states (GOCP_BUILD_SECTOR).
//
// H (Eq. 2 -> 3) and every pool generator conserve the numbers of alpha and
// beta electrons, so the reference state, every Taylor step (Eq. 5, 6), H psi
// (Eq. 3), the energy (Eq. 1), the gradients (Eq. 4) and the adjoint sweep
// stay in the span of the determinants with the reference state's counts.
// A sector-layout state stores only those D amplitudes (SecDev: row r =
// rank_a * C(no, nb) + rank_b).  A Pauli group with mask x maps the
// determinant with occupation n to n ^ u, u = beta^-1 x (the mapping's
// inverse encoding matrix), so the source row of every term is two rank
// lookups away, and a source outside the sector contributes nothing.  The
// coefficients D_g(k) are evaluated at the qubit basis state k of the output
// row exactly as in the full layout (LUT form, paired or plain term lists,
// compensated diagonal), so the numbers on the sector are those of the full
// layout there.
#include <algorithm>
#include <cstring>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace gocp {

// Per-generator pair lists: the pairs {r, r2} (r the base side, bit s of
// its qubit state clear) that generator k touches inside the sector are
// pairs[off[k] .. off[k+1]) (pool order), found once at build time.
struct SectorTables {
  SecDev s;
  int32_t ref_row = 0;
  const uint2* pairs = nullptr;
  const int64_t* off = nullptr;     // device, M + 1
  int64_t max_pairs = 0;            // largest list
  // H on the sector as CSR (built when its couplings are real and it fits
  // kCsrMaxBytes and a quarter of the free device memory; else H psi stays
  // matrix-free): rows ptr[r] .. ptr[r+1]
  const int64_t* csr_ptr = nullptr;
  const uint32_t* csr_col = nullptr;
  const void* csr_val = nullptr;
  const double* csr_diag = nullptr;
  int64_t csr_nnz = 0;
  std::vector<void*> allocs;
};

namespace {

constexpr int kSecThreads = 256;
constexpr int kSecChunk = 64;          // LUT groups staged per chunk (H psi)
constexpr int kSecOps = 16;            // generators per block (pool gradients)
constexpr int kSecRowsPerThread = 16;  // pairs per thread per generator (pool gradients)
constexpr size_t kCsrMaxBytes = (size_t)64 << 30;  // largest CSR form of H built (and <= 1/4 of free memory)

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int grid_rows(int64_t rows, int sm_count, int per_sm) {
  const int64_t need = (rows + kSecThreads - 1) / kSecThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sm_count * per_sm));
}

template <typename R>
__device__ __forceinline__ void kahan(R& s, R& c, R v) {
  if (sizeof(R) == 4) {
    const R y = v - c, t = s + y;
    c = (t - s) - y;
    s = t;
  } else {
    s += v;
  }
}

// psi = row ref; block 0 also writes coefs[6j + m] = theta_j^m / m!.
template <typename R>
__global__ void __launch_bounds__(kSecThreads)
k_sec_setup(C_t<R>* psi, int32_t D, int32_t ref, const double* theta, int n_ops, double* coefs) {
  if (psi)
    for (int32_t r = blockIdx.x * kSecThreads + threadIdx.x; r < D; r += gridDim.x * kSecThreads)
      psi[r] = cmake<R>(r == ref ? R(1) : R(0), R(0));
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < n_ops; j += kSecThreads) {
      double th = theta[j], c = 1.0;
      coefs[6 * j] = 1.0;
      for (int m = 1; m <= 5; ++m) {
        c = c * th / (double)m;
        coefs[6 * j + m] = c;
      }
    }
}

// One Taylor step (Eq. 5, 6) of generator ops[j] in LUT form over its pair
// list (the pairs it touches inside the sector; elsewhere T = I).
template <typename R>
__global__ void __launch_bounds__(kSecThreads)
k_sec_taylor(SecDev s, DevTables tb, const uint2* pairs, const int64_t* off, const int32_t* ops,
             const double* coefs, int j, C_t<R>* psi, int32_t* err) {
  chain_step_begin();
  const int op = ops[j];
  if (op < 0 || op >= tb.M) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, 1);
    return;
  }
  const LutDev<R>& L = ((const LutDev<R>*)tb.plut)[op];   // read in place (lut is indexed at run time)
  R c[6];
  step_coefs<R>(coefs, j, c);
  const uint32_t phx = L.fx & 7u, sgx = (L.fx >> 3) & 1u;
  const int64_t q0 = off[op], np = off[op + 1] - q0;
  for (int64_t i = blockIdx.x * kSecThreads + threadIdx.x; i < np; i += (int64_t)gridDim.x * kSecThreads) {
    const uint2 pr = pairs[q0 + i];
    const uint32_t k = s.kq[pr.x];
    const uint32_t ph = lut_phi(L, k);
    const R l1 = L.lut[ph], l2 = L.lut[ph ^ phx];
    const uint32_t sg = __popc(k & L.z0) & 1u;
    const R d1 = sg ? -l1 : l1, d2 = (sg ^ sgx) ? -l2 : l2;
    C_t<R> v1 = psi[pr.x], v2 = psi[pr.y];
    if constexpr (sizeof(R) == 8) {
      // complex128: the same polynomial through A^2 = mu I on the pair (see
      // taylor_pair_at in kernels.cu)
      const R mu = d1 * d2, mu2 = mu * mu;
      const R cc = c[0] + c[2] * mu + c[4] * mu2;
      const R sc = c[1] + c[3] * mu + c[5] * mu2;
      const R sd1 = sc * d1, sd2 = sc * d2;
      psi[pr.x] = cmake<R>(cc * v1.x + sd1 * v2.x, cc * v1.y + sd1 * v2.y);
      psi[pr.y] = cmake<R>(cc * v2.x + sd2 * v1.x, cc * v2.y + sd2 * v1.y);
      continue;
    }
    C_t<R> s1 = v1, s2 = v2, e1 = cmake<R>(0, 0), e2 = cmake<R>(0, 0);
#pragma unroll
    for (int m = 1; m <= 5; ++m) {
      const C_t<R> n1 = cscale<R>(v2, d1), n2 = cscale<R>(v1, d2);   // (A v)[k] = D(k) v[k ^ x]
      v1 = n1;
      v2 = n2;
      kahan<R>(s1.x, e1.x, v1.x * c[m]);
      kahan<R>(s1.y, e1.y, v1.y * c[m]);
      kahan<R>(s2.x, e2.x, v2.x * c[m]);
      kahan<R>(s2.y, e2.y, v2.y * c[m]);
    }
    psi[pr.x] = csub<R>(s1, e1);
    psi[pr.y] = csub<R>(s2, e2);
  }
}

// D(k) of one term-list group, real and imaginary parts: the paired form
// (1 + sigma (-1)^popc(k & delta)) E(k) when the group pairs, else the plain
// sums.
template <typename R>
__device__ __forceinline__ void sec_term_d(const DevTables& tb, int g, uint32_t k, R* dr, R* di) {
  const R* w = (const R*)tb.sp_w;
  const int tb0 = tb.sp_off[g], tm = tb.sp_mid[g], te = tb.sp_off[g + 1];
  const uint32_t delta = tb.sp_delta[g];
  R a = 0, b = 0;
  if (delta) {
    const bool odd = __popc(k & delta) & 1;
    if (tb.sp_neg[g] ? !odd : odd) {
      *dr = R(0);
      *di = R(0);
      return;
    }
    for (int t = tb0; t < tm; ++t) a += (__popc(k & tb.sp_z[t]) & 1) ? -w[t] : w[t];
    *dr = R(2) * a;
    *di = R(0);
    return;
  }
  for (int t = tb0; t < tm; ++t) a += (__popc(k & tb.sp_z[t]) & 1) ? -w[t] : w[t];
  for (int t = tm; t < te; ++t) b += (__popc(k & tb.sp_z[t]) & 1) ? -w[t] : w[t];
  *dr = a;
  *di = b;
}

// The off-diagonal couplings of one output row (qubit state k, occupation
// n): f(r2, dr, di) for every group whose source row r2 is in the sector and
// whose D(k) = dr + i di is not zero -- LUT groups first (staged kSecChunk at
// a time in shared memory, so every thread of the block must call this),
// then the term-list groups.
template <typename R, typename F>
__device__ __forceinline__ void sec_walk(const SecDev& s, const DevTables& tb, HLut<R>* s_l, uint32_t* s_u,
                                         bool live, uint32_t k, uint32_t n, F&& f) {
  const HLut<R>* hl = (const HLut<R>*)tb.hlut;
  for (int g0 = 0; g0 < tb.GL; g0 += kSecChunk) {
    const int cn = min(kSecChunk, tb.GL - g0);
    __syncthreads();
    for (int q = threadIdx.x; q < cn; q += kSecThreads) {
      s_l[q] = hl[g0 + q];
      s_u[q] = tb.hu[g0 + q];
    }
    __syncthreads();
    if (!live) continue;
    for (int q = 0; q < cn; ++q) {
      uint32_t r2;
      if (!sec_row(s, n, s_u[q], &r2)) continue;
      const HLut<R>& L = s_l[q];
      const uint32_t code = (uint32_t)(__popc(k & L.v0) & 1) | ((uint32_t)(__popc(k & L.v1) & 1) << 1) |
                            ((uint32_t)(__popc(k & L.v2) & 1) << 2) | ((uint32_t)(__popc(k & L.z0) & 1) << 3);
      const R val = L.lut16[code];
      if (val != R(0)) f(r2, val, R(0));
    }
  }
  if (!live) return;
  for (int g = 0; g < tb.G; ++g) {
    uint32_t r2;
    if (!sec_row(s, n, tb.gu[g], &r2)) continue;
    R dr, di;
    sec_term_d<R>(tb, g, k, &dr, &di);
    if (dr != R(0) || di != R(0)) f(r2, dr, di);
  }
}

// H psi (Eq. 3) on the sector, one output row per thread, with the FP64
// energy epilogue (Eq. 1) when partials is set: scal[1] = <psi|psi>,
// scal[2] = Re<psi|H' psi>, scal[0] = E = identity + scal[2] / scal[1].
template <typename R>
__global__ void __launch_bounds__(kSecThreads)
k_sec_apply(SecDev s, DevTables tb, const C_t<R>* __restrict__ psi, C_t<R>* __restrict__ out, double identity,
            double* partials, unsigned int* counter, double* scal) {
  __shared__ HLut<R> s_l[kSecChunk];
  __shared__ uint32_t s_u[kSecChunk];
  __shared__ double tot[2];
  const R* dw = (const R*)tb.dw;
  const R idr = (R)identity;
  double v[2] = {0.0, 0.0};
  for (int32_t base = blockIdx.x * kSecThreads; base < s.D; base += gridDim.x * kSecThreads) {
    const int32_t r = base + threadIdx.x;
    const bool live = r < s.D;
    const uint32_t k = live ? s.kq[r] : 0u, n = live ? s.occ[r] : 0u;
    C_t<R> acc = cmake<R>(0, 0);
    sec_walk<R>(s, tb, s_l, s_u, live, k, n, [&](uint32_t r2, R dr, R di) {
      const C_t<R> p = psi[r2];
      acc.x += dr * p.x - di * p.y;
      acc.y += dr * p.y + di * p.x;
    });
    if (live) {
      // diagonal group (compensated real part) and identity
      R d = 0, dc = 0, e = 0;
      for (int t = 0; t < tb.nd_mid; ++t) kahan<R>(d, dc, (__popc(k & tb.dz[t]) & 1) ? -dw[t] : dw[t]);
      for (int t = tb.nd_mid; t < tb.nd; ++t) e += (__popc(k & tb.dz[t]) & 1) ? -dw[t] : dw[t];
      const C_t<R> p = psi[r];
      const double pp = (double)p.x * p.x + (double)p.y * p.y;
      v[0] += pp;
      v[1] += (double)p.x * acc.x + (double)p.y * acc.y + ((double)d - (double)dc) * pp;
      const R d0 = d - dc + idr;
      out[r] = cmake<R>(acc.x + d0 * p.x - e * p.y, acc.y + d0 * p.y + e * p.x);
    }
  }
  if (partials && block_grid_sum<2, kSecThreads>(v, partials, counter, gridDim.x, blockIdx.x, scal + 1, tot)) {
    if (threadIdx.x == 0) scal[0] = identity + tot[1] / tot[0];
  }
}

// The sector's H as a CSR matrix (real couplings only): FILL = false writes
// the row counts, FILL = true the columns and values in walk order at
// ptr[r] and the diagonal D_0(k) (without the identity) summed in FP64.
template <typename R, bool FILL>
__global__ void __launch_bounds__(kSecThreads)
k_sec_csr(SecDev s, DevTables tb, int64_t* ptr_or_count, uint32_t* cols, R* vals, double* diag) {
  __shared__ HLut<R> s_l[kSecChunk];
  __shared__ uint32_t s_u[kSecChunk];
  const R* dw = (const R*)tb.dw;
  for (int32_t base = blockIdx.x * kSecThreads; base < s.D; base += gridDim.x * kSecThreads) {
    const int32_t r = base + threadIdx.x;
    const bool live = r < s.D;
    const uint32_t k = live ? s.kq[r] : 0u, n = live ? s.occ[r] : 0u;
    int64_t pos = (FILL && live) ? ptr_or_count[r] : 0;
    sec_walk<R>(s, tb, s_l, s_u, live, k, n, [&](uint32_t r2, R dr, R) {
      if (FILL) {
        cols[pos] = r2;
        vals[pos] = dr;
      }
      ++pos;
    });
    if (!live) continue;
    if (FILL) {
      double d = 0.0;
      for (int t = 0; t < tb.nd_mid; ++t) d += (__popc(k & tb.dz[t]) & 1) ? -(double)dw[t] : (double)dw[t];
      diag[r] = d;
    } else {
      ptr_or_count[r] = pos;
    }
  }
}

// H psi from the CSR form, one warp per row, with the energy epilogue.
template <typename R>
__global__ void __launch_bounds__(kSecThreads)
k_sec_spmv(int32_t D, const int64_t* __restrict__ ptr, const uint32_t* __restrict__ cols, const R* __restrict__ vals,
           const double* __restrict__ diag, const C_t<R>* __restrict__ psi, C_t<R>* __restrict__ out,
           double identity, double* partials, unsigned int* counter, double* scal) {
  __shared__ double tot[2];
  const int lane = threadIdx.x & 31;
  const int32_t warps = gridDim.x * (kSecThreads / 32);
  double v[2] = {0.0, 0.0};
  for (int32_t r = blockIdx.x * (kSecThreads / 32) + (threadIdx.x >> 5); r < D; r += warps) {
    const int64_t q0 = ptr[r], q1 = ptr[r + 1];
    R ax = 0, ay = 0, cx = 0, cy = 0;   // compensated lane sums (FP32)
    for (int64_t q = q0 + lane; q < q1; q += 32) {
      const R w = vals[q];
      const C_t<R> p = psi[cols[q]];
      kahan<R>(ax, cx, w * p.x);
      kahan<R>(ay, cy, w * p.y);
    }
    ax -= cx;
    ay -= cy;
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) {
      const C_t<R> p = psi[r];
      const double pp = (double)p.x * p.x + (double)p.y * p.y, d = diag[r];
      v[0] += pp;
      v[1] += (double)p.x * ax + (double)p.y * ay + d * pp;
      const R d0 = (R)(d + identity);
      out[r] = cmake<R>(ax + d0 * p.x, ay + d0 * p.y);
    }
  }
  if (partials && block_grid_sum<2, kSecThreads>(v, partials, counter, gridDim.x, blockIdx.x, scal + 1, tot)) {
    if (threadIdx.x == 0) scal[0] = identity + tot[1] / tot[0];
  }
}

// lambda = (H psi - E psi) / <psi|psi> in place (E, <psi|psi> = scal[0..1]).
template <typename R>
__global__ void __launch_bounds__(kSecThreads)
k_sec_residual(const C_t<R>* psi, C_t<R>* lam, int32_t D, const double* scal) {
  const R er = (R)scal[0], ir = (R)(1.0 / scal[1]);
  for (int32_t r = blockIdx.x * kSecThreads + threadIdx.x; r < D; r += gridDim.x * kSecThreads) {
    const C_t<R> h = lam[r], p = psi[r];
    lam[r] = cmake<R>((h.x - er * p.x) * ir, (h.y - er * p.y) * ir);
  }
}

// Pool gradients (Eq. 4) over the pair lists: blockIdx.y picks kSecOps
// generators in GOCP family order, blockIdx.x a slice of per_block pairs of
// each; per pair {k, k ^ x}
//   Re<H psi|A psi> += D(k) Re(conj(h_k) psi_{k^x}) + D(k^x) Re(conj(h_{k^x}) psi_k).
// part[i * nbx + blockIdx.x] = this block's sum for generator i (family order).
template <typename R>
__global__ void __launch_bounds__(kSecThreads)
k_sec_pool_grad(SecDev s, DevTables tb, const uint2* pairs, const int64_t* off, const C_t<R>* __restrict__ psi,
                const C_t<R>* __restrict__ hpsi, double* part, int nbx, int64_t per_block) {
  __shared__ double s_red[kSecThreads / 32];
  const int first = blockIdx.y * kSecOps;
  const int nops = min(kSecOps, tb.M - first);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 0; o < nops; ++o) {
    const int op = tb.porder[first + o];
    const LutDev<R>& L = ((const LutDev<R>*)tb.plut)[op];
    const uint32_t phx = L.fx & 7u, sgx = (L.fx >> 3) & 1u;
    const int64_t q0 = off[op] + (int64_t)blockIdx.x * per_block;
    const int64_t q1 = min(off[op + 1], q0 + per_block);
    R acc = 0, cmp = 0;
    for (int64_t q = q0 + threadIdx.x; q < q1; q += kSecThreads) {
      const uint2 pr = pairs[q];
      const uint32_t k = s.kq[pr.x];
      const uint32_t ph = lut_phi(L, k);
      const R l1 = L.lut[ph], l2 = L.lut[ph ^ phx];
      const uint32_t sg = __popc(k & L.z0) & 1u;
      const C_t<R> h1 = hpsi[pr.x], h2 = hpsi[pr.y], p1 = psi[pr.x], p2 = psi[pr.y];
      const R val = (sg ? -l1 : l1) * (h1.x * p2.x + h1.y * p2.y) +
                    ((sg ^ sgx) ? -l2 : l2) * (h2.x * p1.x + h2.y * p1.y);
      kahan<R>(acc, cmp, val);
    }
    // the warp's sum in R (FP64 is a slow pipe here), the block's in FP64
    const R wv = warp_total<R>(acc - cmp);
    if (lane == 0) s_red[warp] = (double)wv;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kSecThreads / 32; ++w) t += s_red[w];
      part[(size_t)(first + o) * nbx + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// Backward step j of the adjoint sweep (see the full-layout k_adjoint) over
// the pair list of ops[j]: psi <- T^-1 psi exactly, dE_j += 2 Re <lambda|T' psi>,
// lambda <- T^dagger lambda.
template <typename R>
__global__ void __launch_bounds__(kSecThreads)
k_sec_adjoint(SecDev s, DevTables tb, const uint2* pairs, const int64_t* off, const int32_t* ops,
              const double* coefs, int j, C_t<R>* psi, C_t<R>* lam, double* partials, unsigned int* counter,
              double* dtheta, int32_t* err) {
  __shared__ double tot[1];
  chain_step_begin();
  const int op = ops[j];
  if (op < 0 || op >= tb.M) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicOr(err, 1);
      dtheta[j] = 0.0;
    }
    return;
  }
  const LutDev<R>& L = ((const LutDev<R>*)tb.plut)[op];   // read in place (lut is indexed at run time)
  R c[6];
  step_coefs<R>(coefs, j, c);
  const uint32_t phx = L.fx & 7u, sgx = (L.fx >> 3) & 1u;
  const int64_t q0 = off[op], np = off[op + 1] - q0;
  // this thread's part of dE_j, compensated in R; warps then sum in R and
  // blocks in FP64 (FP64 is a slow pipe on this part)
  R acc = R(0), cmp = R(0);
  for (int64_t i = blockIdx.x * kSecThreads + threadIdx.x; i < np; i += (int64_t)gridDim.x * kSecThreads) {
    const uint2 pr = pairs[q0 + i];
    const uint32_t k = s.kq[pr.x];
    const uint32_t ph = lut_phi(L, k);
    const R l1 = L.lut[ph], l2 = L.lut[ph ^ phx];
    const uint32_t sg = __popc(k & L.z0) & 1u;
    const R d1 = sg ? -l1 : l1, d2 = (sg ^ sgx) ? -l2 : l2;
    const R mu = d1 * d2, mu2 = mu * mu;
    const R cc = c[0] + c[2] * mu + c[4] * mu2;
    const R sc = c[1] + c[3] * mu + c[5] * mu2;
    const R cd = c[1] * mu + c[3] * mu2;
    const R inv = R(1) / (cc * cc - sc * sc * mu);
    const R sd1 = sc * d1, sd2 = sc * d2;
    const C_t<R> u1 = psi[pr.x], u2 = psi[pr.y];
    const C_t<R> q1 = cscale<R>(csub<R>(cscale<R>(u1, cc), cscale<R>(u2, sd1)), inv);
    const C_t<R> q2 = cscale<R>(csub<R>(cscale<R>(u2, cc), cscale<R>(u1, sd2)), inv);
    const C_t<R> t1 = cadd<R>(cscale<R>(q1, cd), cscale<R>(q2, cc * d1));
    const C_t<R> t2 = cadd<R>(cscale<R>(q2, cd), cscale<R>(q1, cc * d2));
    const C_t<R> l1v = lam[pr.x], l2v = lam[pr.y];
    kahan<R>(acc, cmp, R(2) * (l1v.x * t1.x + l1v.y * t1.y + l2v.x * t2.x + l2v.y * t2.y));
    psi[pr.x] = q1;
    psi[pr.y] = q2;
    lam[pr.x] = cadd<R>(cscale<R>(l1v, cc), cscale<R>(l2v, sd2));
    lam[pr.y] = cadd<R>(cscale<R>(l1v, sd1), cscale<R>(l2v, cc));
  }
  const double v[1] = {(double)warp_total<R>(acc - cmp)};
  block_grid_sum<1, kSecThreads, true>(v, partials, counter, gridDim.x, blockIdx.x, dtheta + j, tot);
}

template <typename R>
__global__ void __launch_bounds__(kSecThreads)
k_sec_scatter(const C_t<R>* __restrict__ psi, C_t<R>* __restrict__ full, const uint32_t* kq, int32_t D) {
  for (int32_t r = blockIdx.x * kSecThreads + threadIdx.x; r < D; r += gridDim.x * kSecThreads) full[kq[r]] = psi[r];
}

template <typename R>
__global__ void __launch_bounds__(kSecThreads)
k_sec_gather(const C_t<R>* __restrict__ full, C_t<R>* __restrict__ psi, const uint32_t* kq, int32_t D) {
  for (int32_t r = blockIdx.x * kSecThreads + threadIdx.x; r < D; r += gridDim.x * kSecThreads) psi[r] = full[kq[r]];
}

// Whether row r is the base of a pair generator L touches inside the
// sector; *r2 = the partner row.
template <typename R>
__device__ __forceinline__ bool sec_pair(const SecDev& s, const LutDev<R>& L, uint32_t u, int32_t r, uint32_t* r2) {
  const uint32_t k = s.kq[r];
  if ((k >> L.s) & 1u) return false;
  if (!sec_row(s, s.occ[r], u, r2)) return false;
  const uint32_t ph = lut_phi(L, k);
  return L.lut[ph] != R(0) || L.lut[ph ^ (L.fx & 7u)] != R(0);
}

// counts[k * nchunk + c] = pairs of generator k (pool order) based in rows
// [256 c, 256 c + 256).
template <typename R>
__global__ void __launch_bounds__(kSecThreads) k_sec_pair_count(SecDev s, DevTables tb, int nchunk, int64_t* counts) {
  __shared__ int wsum[kSecThreads / 32];
  const int k = blockIdx.y;
  const LutDev<R>& L = ((const LutDev<R>*)tb.plut)[k];
  const uint32_t u = tb.pu[k];
  for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
    const int32_t r = c * kSecThreads + threadIdx.x;
    uint32_t r2;
    const bool hit = r < s.D && sec_pair<R>(s, L, u, r, &r2);
    const int n = __popc(__ballot_sync(0xffffffffu, hit));
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < kSecThreads / 32; ++w) t += wsum[w];
      counts[(int64_t)k * nchunk + c] = t;
    }
    __syncthreads();
  }
}

// Writes the pairs in row order at base[k * nchunk + c] (exclusive prefix
// sums of the counts).
template <typename R>
__global__ void __launch_bounds__(kSecThreads)
k_sec_pair_fill(SecDev s, DevTables tb, int nchunk, const int64_t* base, uint2* pairs) {
  __shared__ int wsum[kSecThreads / 32];
  const int k = blockIdx.y;
  const LutDev<R>& L = ((const LutDev<R>*)tb.plut)[k];
  const uint32_t u = tb.pu[k];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
    const int32_t r = c * kSecThreads + threadIdx.x;
    uint32_t r2 = 0;
    const bool hit = r < s.D && sec_pair<R>(s, L, u, r, &r2);
    const uint32_t bal = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    if (hit) {
      const int64_t at = base[(int64_t)k * nchunk + c] + before + __popc(bal & ((1u << lane) - 1u));
      pairs[at] = make_uint2((uint32_t)r, r2);
    }
    __syncthreads();
  }
}

template <typename T>
int sec_upload(SectorTables& st, T** p, const std::vector<T>& h, size_t& bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(h.size(), 1) * sizeof(T));
  if (e != cudaSuccess) return cuda_status(e, "cudaMalloc (sector tables)");
  st.allocs.push_back(q);
  bytes += h.size() * sizeof(T);
  *p = (T*)q;
  if (h.empty()) return GOCP_OK;
  return cuda_status(cudaMemcpy(q, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice), "cudaMemcpy (sector)");
}

int check_sector(const Problem& p) {
  if (!p.sector || !p.sec) return fail(GOCP_EINVAL, "problem is not in the sector layout");
  return GOCP_OK;
}

int sm_of(Problem& p) { return std::max(p.sm_count, 1); }

template <typename R>
int sec_apply_t(Problem& p, const void* psi, void* hpsi, bool energy, cudaStream_t st) {
  size_t nd = 0;
  double* scratch = scratch_ptr(p, &nd);
  if (p.sec->csr_val) {
    const int32_t D = p.sec->s.D;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>({(D + 7) / 8, (int64_t)sm_of(p) * 16, (int64_t)nd / 2}));
    k_sec_spmv<R><<<grid, kSecThreads, 0, st>>>(D, p.sec->csr_ptr, p.sec->csr_col, (const R*)p.sec->csr_val,
                                                p.sec->csr_diag, (const C_t<R>*)psi, (C_t<R>*)hpsi, p.identity,
                                                energy ? scratch : nullptr, counters_ptr(p), scalars_ptr(p));
    count_launches(1);
    return cuda_status(cudaGetLastError(), "k_sec_spmv");
  }
  const int grid = std::min<int>(grid_rows(p.sector_dim, sm_of(p), 8), (int)(nd / 2));
  k_sec_apply<R><<<grid, kSecThreads, 0, st>>>(p.sec->s, dev_tables(p), (const C_t<R>*)psi, (C_t<R>*)hpsi,
                                               p.identity, energy ? scratch : nullptr, counters_ptr(p),
                                               scalars_ptr(p));
  count_launches(1);
  return cuda_status(cudaGetLastError(), "k_sec_apply");
}

int pair_grid(Problem& p, int per_sm) {
  const int64_t need = (p.sec->max_pairs + kSecThreads - 1) / kSecThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sm_of(p) * per_sm));
}

template <typename R>
int sec_taylor_t(Problem& p, const int32_t* d_ops, int n_ops, void* psi, cudaStream_t st) {
  const int grid = pair_grid(p, 8);
  SecDev sd = p.sec->s;
  DevTables tb = dev_tables(p);
  const uint2* pairs = p.sec->pairs;
  const int64_t* off = p.sec->off;
  const double* coefs = coefs_ptr(p);
  int j = 0;
  C_t<R>* ps_ = (C_t<R>*)psi;
  int32_t* err = err_ptr(p);
  void* args[] = {&sd, &tb, &pairs, &off, &d_ops, &coefs, &j, &ps_, &err};
  // sd and tb are fixed for the problem's lifetime: not part of the chain key
  const size_t sizes[] = {0, 0, sizeof(pairs), sizeof(off), sizeof(d_ops), sizeof(coefs), sizeof(j), sizeof(ps_),
                          sizeof(err)};
  ProfScope ps(GOCP_KERNEL_TAYLOR, st, n_ops);
  int rc = launch_chain(p, (const void*)k_sec_taylor<R>, grid, kSecThreads, n_ops, false, args, sizes, 9, 6, st);
  if (rc) return rc;
  return cuda_status(cudaGetLastError(), "k_sec_taylor");
}

template <typename R>
int sec_pool_t(Problem& p, const void* psi, const void* hpsi, double* d_grads, cudaStream_t st) {
  const DevTables& tb = dev_tables(p);
  const int M = tb.M;
  if (M == 0) return GOCP_OK;
  const int nchunks = (M + kSecOps - 1) / kSecOps;
  size_t nd = 0;
  double* scratch = scratch_ptr(p, &nd);
  const int64_t per = kSecThreads * kSecRowsPerThread;
  int nbx = (int)std::max<int64_t>(1, (p.sec->max_pairs + per - 1) / per);
  nbx = std::max(1, std::min<int>(nbx, (int)(nd / ((size_t)nchunks * kSecOps))));
  const int64_t per_block = (p.sec->max_pairs + nbx - 1) / nbx;
  {
    ProfScope ps(GOCP_KERNEL_POOL_GRAD, st);
    k_sec_pool_grad<R><<<dim3(nbx, nchunks), kSecThreads, 0, st>>>(p.sec->s, tb, p.sec->pairs, p.sec->off,
                                                                   (const C_t<R>*)psi, (const C_t<R>*)hpsi, scratch,
                                                                   nbx, std::max<int64_t>(per_block, 1));
  }
  count_launches(1);
  int rc = cuda_status(cudaGetLastError(), "k_sec_pool_grad");
  if (rc) return rc;
  return pool_finish(p, scratch, nbx, d_grads, st);
}

template <typename R>
int sec_adjoint_t(Problem& p, const int32_t* d_ops, int n_ops, void* psi, void* lam, double* d_dE, cudaStream_t st) {
  const int32_t D = p.sec->s.D;
  size_t nd = 0;
  double* scratch = scratch_ptr(p, &nd);
  k_sec_residual<R><<<grid_rows(D, sm_of(p), 8), kSecThreads, 0, st>>>((const C_t<R>*)psi, (C_t<R>*)lam, D,
                                                                       scalars_ptr(p));
  count_launches(1);   // k_sec_residual
  const int grid = std::min<int>(pair_grid(p, 2), (int)nd);
  SecDev sd = p.sec->s;
  DevTables tb = dev_tables(p);
  const uint2* pairs = p.sec->pairs;
  const int64_t* off = p.sec->off;
  const double* coefs = coefs_ptr(p);
  int j = 0;
  C_t<R>* ps_ = (C_t<R>*)psi;
  C_t<R>* ls_ = (C_t<R>*)lam;
  unsigned int* counter = counters_ptr(p) + 2;
  int32_t* err = err_ptr(p);
  void* args[] = {&sd, &tb, &pairs, &off, &d_ops, &coefs, &j, &ps_, &ls_, &scratch, &counter, &d_dE, &err};
  const size_t sizes[] = {0, 0, sizeof(pairs), sizeof(off), sizeof(d_ops), sizeof(coefs), sizeof(j), sizeof(ps_),
                          sizeof(ls_), sizeof(scratch), sizeof(counter), sizeof(d_dE), sizeof(err)};
  ProfScope ps(GOCP_KERNEL_ADJOINT, st, n_ops);
  int rc = launch_chain(p, (const void*)k_sec_adjoint<R>, grid, kSecThreads, n_ops, true, args, sizes, 13, 6, st);
  if (rc) return rc;
  return cuda_status(cudaGetLastError(), "k_sec_adjoint");
}

// Builds the CSR form of H on the sector (see SectorTables) when every
// coupling is real and it fits kCsrMaxBytes and a quarter of the free device
// memory; leaves it absent otherwise.
template <typename R>
int build_csr(Problem& p, SectorTables& st, size_t& bytes) {
  for (size_t t = 0; t < p.H.size(); ++t)
    if (p.H.phase[t] & 1) return GOCP_OK;   // an imaginary weight: stay matrix-free
  const DevTables& tb = dev_tables(p);
  const int32_t D = st.s.D;
  int64_t* dptr = nullptr;
  cudaError_t e = cudaMalloc(&dptr, ((size_t)D + 1) * sizeof(int64_t));
  if (e != cudaSuccess) return cuda_status(e, "cudaMalloc (CSR rows)");
  const int grid = grid_rows(D, sm_of(p), 8);
  k_sec_csr<R, false><<<grid, kSecThreads>>>(st.s, tb, dptr, nullptr, nullptr, nullptr);
  count_launches(1);
  std::vector<int64_t> ptr((size_t)D + 1, 0);
  int rc = cuda_status(cudaMemcpy(ptr.data(), dptr, (size_t)D * sizeof(int64_t), cudaMemcpyDeviceToHost),
                       "copy CSR counts");
  int64_t nnz = 0;
  for (int32_t r = 0; r < D; ++r) {
    const int64_t c = ptr[r];
    ptr[r] = nnz;
    nnz += c;
  }
  ptr[D] = nnz;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
  const size_t need = (size_t)nnz * (4 + sizeof(R));
  if (rc || need > kCsrMaxBytes || need > free_b / 4) {
    cudaGetLastError();
    cudaFree(dptr);
    return rc;
  }
  st.allocs.push_back(dptr);
  uint32_t* dcol = nullptr;
  R* dval = nullptr;
  double* ddiag = nullptr;
  if ((rc = cuda_status(cudaMemcpy(dptr, ptr.data(), ptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice),
                        "upload CSR rows")))
    return rc;
  if ((e = cudaMalloc(&dcol, std::max<int64_t>(nnz, 1) * sizeof(uint32_t))) != cudaSuccess)
    return cuda_status(e, "cudaMalloc (CSR columns)");
  st.allocs.push_back(dcol);
  if ((e = cudaMalloc(&dval, std::max<int64_t>(nnz, 1) * sizeof(R))) != cudaSuccess)
    return cuda_status(e, "cudaMalloc (CSR values)");
  st.allocs.push_back(dval);
  if ((e = cudaMalloc(&ddiag, (size_t)D * sizeof(double))) != cudaSuccess)
    return cuda_status(e, "cudaMalloc (CSR diagonal)");
  st.allocs.push_back(ddiag);
  k_sec_csr<R, true><<<grid, kSecThreads>>>(st.s, tb, dptr, dcol, dval, ddiag);
  count_launches(1);
  if ((rc = cuda_status(cudaDeviceSynchronize(), "k_sec_csr"))) return rc;
  bytes += ((size_t)D + 1) * 8 + (size_t)nnz * (4 + sizeof(R)) + (size_t)D * 8;
  st.csr_ptr = dptr;
  st.csr_col = dcol;
  st.csr_val = dval;
  st.csr_diag = ddiag;
  st.csr_nnz = nnz;
  return GOCP_OK;
}

// Builds the per-generator pair lists (see SectorTables).
template <typename R>
int build_pairs(Problem& p, SectorTables& st, size_t& bytes) {
  const DevTables& tb = dev_tables(p);
  const int M = tb.M;
  std::vector<int64_t> off(M + 1, 0);
  if (M == 0) {
    int64_t* doff;
    int rc = sec_upload(st, &doff, off, bytes);
    st.off = doff;
    return rc;
  }
  const int nchunk = (int)((st.s.D + kSecThreads - 1) / kSecThreads);
  const size_t nc = (size_t)M * nchunk;
  int64_t* dcounts = nullptr;
  cudaError_t e = cudaMalloc(&dcounts, nc * sizeof(int64_t));
  if (e != cudaSuccess) return cuda_status(e, "cudaMalloc (pair counts)");
  struct Free {
    int64_t* q;
    ~Free() { cudaFree(q); }
  } hold{dcounts};
  for (int k0 = 0; k0 < M; k0 += 65535) {
    const int mk = std::min(M - k0, 65535);
    DevTables tk = tb;   // generators k0 .. k0 + mk - 1
    tk.plut = (const LutDev<R>*)tb.plut + k0;
    tk.pu = tb.pu + k0;
    k_sec_pair_count<R><<<dim3(std::min(nchunk, 64), mk), kSecThreads>>>(st.s, tk, nchunk, dcounts + (size_t)k0 * nchunk);
  }
  count_launches((M + 65534) / 65535);
  int rc = cuda_status(cudaGetLastError(), "k_sec_pair_count");
  if (rc) return rc;
  std::vector<int64_t> counts(nc), base(nc);
  if ((rc = cuda_status(cudaMemcpy(counts.data(), dcounts, nc * sizeof(int64_t), cudaMemcpyDeviceToHost),
                        "copy pair counts")))
    return rc;
  int64_t total = 0;
  for (int k = 0; k < M; ++k) {
    off[k] = total;
    int64_t mine = 0;
    for (int c = 0; c < nchunk; ++c) {
      base[(size_t)k * nchunk + c] = total + mine;
      mine += counts[(size_t)k * nchunk + c];
    }
    total += mine;
    st.max_pairs = std::max(st.max_pairs, mine);
  }
  off[M] = total;
  int64_t* doff;
  uint2* dpairs = nullptr;
  if ((rc = cuda_status(cudaMemcpy(dcounts, base.data(), nc * sizeof(int64_t), cudaMemcpyHostToDevice),
                        "upload pair offsets")) ||
      (rc = sec_upload(st, &doff, off, bytes)))
    return rc;
  e = cudaMalloc(&dpairs, std::max<int64_t>(total, 1) * sizeof(uint2));
  if (e != cudaSuccess) return cuda_status(e, "cudaMalloc (pair lists)");
  st.allocs.push_back(dpairs);
  bytes += (size_t)total * sizeof(uint2);
  for (int k0 = 0; k0 < M; k0 += 65535) {
    const int mk = std::min(M - k0, 65535);
    DevTables tk = tb;
    tk.plut = (const LutDev<R>*)tb.plut + k0;
    tk.pu = tb.pu + k0;
    k_sec_pair_fill<R><<<dim3(std::min(nchunk, 64), mk), kSecThreads>>>(st.s, tk, nchunk,
                                                                       dcounts + (size_t)k0 * nchunk, dpairs);
  }
  count_launches((M + 65534) / 65535);
  if ((rc = cuda_status(cudaDeviceSynchronize(), "k_sec_pair_fill"))) return rc;
  st.pairs = dpairs;
  st.off = doff;
  return GOCP_OK;
}

}  // namespace

int upload_sector(Problem& p) {
  if (!p.sector) return GOCP_OK;
  if (p.n_elec < 0 || p.mapping < 0) return fail(GOCP_EINVAL, "sector layout needs a problem built from integrals");
  const int no = p.n_qubits / 2;
  if (no > 16) return fail(GOCP_EINVAL, "sector layout supports at most 16 spatial orbitals");
  const int na = (p.n_elec + 1) / 2, nb = p.n_elec / 2;
  std::vector<uint32_t> sa, sb, rank_a((size_t)1 << no, 0u), rank_b((size_t)1 << no, 0u);
  for (uint32_t m = 0; m < (1u << no); ++m) {
    if (__builtin_popcount(m) == na) {
      rank_a[m] = (uint32_t)sa.size();
      sa.push_back(m);
    }
    if (__builtin_popcount(m) == nb) {
      rank_b[m] = (uint32_t)sb.size();
      sb.push_back(m);
    }
  }
  const int64_t D = (int64_t)sa.size() * (int64_t)sb.size();
  if (D <= 0 || D > ((int64_t)1 << 30)) return fail(GOCP_EINVAL, "sector dimension out of range");
  const Encoding enc = make_encoding(p.mapping, p.n_qubits);
  std::vector<uint32_t> occ((size_t)D), kq((size_t)D);
  for (size_t ia = 0; ia < sa.size(); ++ia)
    for (size_t ib = 0; ib < sb.size(); ++ib) {
      const size_t r = ia * sb.size() + ib;
      uint32_t spin = 0;   // spin-orbital 2q + s
      for (int q = 0; q < no; ++q)
        spin |= (((sa[ia] >> q) & 1u) << (2 * q)) | (((sb[ib] >> q) & 1u) << (2 * q + 1));
      occ[r] = sa[ia] | (sb[ib] << 16);
      kq[r] = enc.encode(spin);
    }
  SectorTables* st = new SectorTables();
  p.sec = st;
  size_t bytes = 0;
  uint32_t *docc, *dkq, *dra, *drb;
  int rc;
  if ((rc = sec_upload(*st, &docc, occ, bytes)) || (rc = sec_upload(*st, &dkq, kq, bytes)) ||
      (rc = sec_upload(*st, &dra, rank_a, bytes)) || (rc = sec_upload(*st, &drb, rank_b, bytes)))
    return rc;
  st->s.D = (int32_t)D;
  st->s.no = no;
  st->s.na = na;
  st->s.nb = nb;
  st->s.cb = (uint32_t)sb.size();
  st->s.occ = docc;
  st->s.kq = dkq;
  st->s.rank_a = dra;
  st->s.rank_b = drb;
  // the reference state: the na lowest alpha and nb lowest beta orbitals
  st->ref_row = (int32_t)(rank_a[(1u << na) - 1u] * sb.size() + rank_b[(1u << nb) - 1u]);
  p.sector_dim = D;
  if ((rc = p.precision == GOCP_C64 ? build_pairs<float>(p, *st, bytes) : build_pairs<double>(p, *st, bytes)))
    return rc;
  if ((rc = p.precision == GOCP_C64 ? build_csr<float>(p, *st, bytes) : build_csr<double>(p, *st, bytes)))
    return rc;
  p.device_bytes += bytes;
  return GOCP_OK;
}

void free_sector(Problem& p) {
  if (!p.sec) return;
  for (void* q : p.sec->allocs) cudaFree(q);
  delete p.sec;
  p.sec = nullptr;
}

int sec_setup(Problem& p, void* psi, const double* d_theta, int n_ops, void* stream) {
  int rc = check_sector(p);
  if (rc || (rc = ensure_stage(p, n_ops))) return rc;
  cudaStream_t st = as_stream(stream);
  const int grid = psi ? grid_rows(p.sector_dim, sm_of(p), 8) : 1;
  if (p.precision == GOCP_C64)
    k_sec_setup<float><<<grid, kSecThreads, 0, st>>>((float2*)psi, p.sec->s.D, p.sec->ref_row, d_theta, n_ops,
                                                     coefs_ptr(p));
  else
    k_sec_setup<double><<<grid, kSecThreads, 0, st>>>((double2*)psi, p.sec->s.D, p.sec->ref_row, d_theta, n_ops,
                                                      coefs_ptr(p));
  count_launches(1);
  return cuda_status(cudaGetLastError(), "k_sec_setup");
}

int sec_taylor_chain(Problem& p, const int32_t* d_ops, int n_ops, void* psi, void* stream) {
  int rc = check_sector(p);
  if (rc || n_ops == 0) return rc;
  return p.precision == GOCP_C64 ? sec_taylor_t<float>(p, d_ops, n_ops, psi, as_stream(stream))
                                 : sec_taylor_t<double>(p, d_ops, n_ops, psi, as_stream(stream));
}

int sec_apply_h(Problem& p, const void* psi, void* hpsi, bool energy, void* stream) {
  int rc = check_sector(p);
  if (rc) return rc;
  ProfScope ps(GOCP_KERNEL_APPLY_H, as_stream(stream));
  return p.precision == GOCP_C64 ? sec_apply_t<float>(p, psi, hpsi, energy, as_stream(stream))
                                 : sec_apply_t<double>(p, psi, hpsi, energy, as_stream(stream));
}

int sec_pool_grads(Problem& p, const void* psi, const void* hpsi, double* d_grads, void* stream) {
  int rc = check_sector(p);
  if (rc || (rc = dev_norm(p, psi, as_stream(stream)))) return rc;   // <psi|psi> -> scalars[1]
  return p.precision == GOCP_C64 ? sec_pool_t<float>(p, psi, hpsi, d_grads, as_stream(stream))
                                 : sec_pool_t<double>(p, psi, hpsi, d_grads, as_stream(stream));
}

int sec_adjoint(Problem& p, const int32_t* d_ops, int n_ops, void* psi, void* lam, double* d_dE, void* stream) {
  int rc = check_sector(p);
  if (rc) return rc;
  return p.precision == GOCP_C64 ? sec_adjoint_t<float>(p, d_ops, n_ops, psi, lam, d_dE, as_stream(stream))
                                 : sec_adjoint_t<double>(p, d_ops, n_ops, psi, lam, d_dE, as_stream(stream));
}

int sec_expand(Problem& p, const void* psi, void* full, void* stream) {
  int rc = check_sector(p);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  const size_t elem = p.precision == GOCP_C64 ? 8u : 16u;
  if ((rc = cuda_status(cudaMemsetAsync(full, 0, ((size_t)1 << p.n_qubits) * elem, st), "clear full state")))
    return rc;
  const int grid = grid_rows(p.sector_dim, sm_of(p), 8);
  if (p.precision == GOCP_C64)
    k_sec_scatter<float><<<grid, kSecThreads, 0, st>>>((const float2*)psi, (float2*)full, p.sec->s.kq, p.sec->s.D);
  else
    k_sec_scatter<double><<<grid, kSecThreads, 0, st>>>((const double2*)psi, (double2*)full, p.sec->s.kq,
                                                        p.sec->s.D);
  count_launches(1);
  return cuda_status(cudaGetLastError(), "k_sec_scatter");
}

int sec_compress(Problem& p, const void* full, void* psi, void* stream) {
  int rc = check_sector(p);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  const int grid = grid_rows(p.sector_dim, sm_of(p), 8);
  if (p.precision == GOCP_C64)
    k_sec_gather<float><<<grid, kSecThreads, 0, st>>>((const float2*)full, (float2*)psi, p.sec->s.kq, p.sec->s.D);
  else
    k_sec_gather<double><<<grid, kSecThreads, 0, st>>>((const double2*)full, (double2*)psi, p.sec->s.kq,
                                                       p.sec->s.D);
  count_launches(1);
  return cuda_status(cudaGetLastError(), "k_sec_gather");
}

}  // namespace gocp
