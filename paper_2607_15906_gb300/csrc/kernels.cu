// sm_103a kernels of the hot path and their launchers.
//
//   apply_body     (H psi)[k] = sum_g D_g(k) psi[k ^ x_g]   (Eq. 3), with the
//                  energy <psi|H psi> / <psi|psi> (Eq. 1) as an FP64 epilogue
//   taylor_body    psi <- sum_{m<=5} theta^m/m! v_m, v_m = A v_{m-1}, evaluated
//                  on each basis pair {b, b^x} in registers (Eq. 5, 6)
//   k_pool_grad    g_k = 2 Re <H psi|A_k psi> / <psi|psi>, all k   (Eq. 4)
//   adjoint_body   one backward step of the adjoint sweep for dE/dtheta
//
// Each body takes (block id, block count) of its own work item, so the same
// code serves one problem (a grid of one item) and the request server (one
// launch over many resident requests of different sizes).
//
// Every reduction is deterministic: each block writes its partial sums and
// the last block to finish (threadfence + counter) adds them in a fixed
// order, so a result does not depend on scheduling or on the batch.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "device.cuh"
#include "internal.h"

namespace gocp {

namespace cg = cooperative_groups;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunkTerms = 2048;    // shared-memory stage of H psi
constexpr int kChunkGroups = 512;
constexpr int kOpsPerBlock = 16;     // pool operators per gradient block
constexpr int kChainBlocksPerSm = 4; // blocks per SM of a Taylor or adjoint step (LUT pools)
constexpr int kStageStrings = 256;   // strings staged per gradient / Taylor block
constexpr int kPairsPerThread = 32;  // pool gradients: pairs per thread per operator
constexpr int kMaxChunks = 8192;     // gradient op chunks (pool <= 131072)
constexpr int kItemBlocksPerSm = 2;  // batched stages: blocks per item per SM
// H psi: resident blocks per SM the register budget must allow (complex64:
// 4, trading a small spill for occupancy, measured faster; complex128: 2)
#ifndef GOCP_APPLY_MIN_BLOCKS_C64
#define GOCP_APPLY_MIN_BLOCKS_C64 4
#endif

struct DeviceTables {
  DevTables t;
  int sm_count = 0;
  std::vector<void*> allocs;
  double* scratch = nullptr;
  size_t scratch_doubles = 0;
  unsigned int* counters = nullptr;  // kMaxChunks + 8
  double* scalars = nullptr;         // [0] E  [1] <psi|psi>  [2] Re<psi|H'psi>
  int32_t* stage_ops = nullptr;
  double* stage_theta = nullptr;
  double* coefs = nullptr;           // 6 Taylor coefficients per ansatz op
  double* dtheta = nullptr;          // stage_cap doubles
  int stage_cap = 0;
  int32_t* err = nullptr;
  int32_t* selected = nullptr;
  double* grads = nullptr;           // pool_size doubles (pool order)
  double* graw = nullptr;            // whole chunks, family order, unscaled
  // live-octet list of the pool-gradient pass and of the scatter H psi
  // kernel (n >= 8)
  LiveOctets live;
  uint32_t* chain_counts = nullptr;   // per-block counts of chain_list
  double* dpart = nullptr;            // stage_cap x adjoint_grid partials of dE/dtheta
};

// ------------------------------------------------------------ reductions

// Adds v[0..NV) over the nblocks blocks of one work item (see block_grid_sum).
template <int NV>
__device__ bool grid_sum(const double (&v)[NV], double* partials, unsigned int* counter,
                         int nblocks, int bid, double* out, double* tot) {
  return block_grid_sum<NV, kThreads>(v, partials, counter, nblocks, bid, out, tot);
}

// ------------------------------------------------------------ setup

// psi = |index>; block 0 also writes the Taylor coefficients
// coefs[6j + m] = theta_j^m / m!, m = 0..5, of every ansatz operator.
template <typename R>
__device__ void setup_body(C_t<R>* psi, int n, uint64_t index, const double* theta, int n_ops,
                           double* coefs, int bid, int nb) {
  const uint64_t dim = 1ull << n;
  if (psi)
    for (uint64_t k = bid * (uint64_t)kThreads + threadIdx.x; k < dim; k += (uint64_t)nb * kThreads)
      psi[k] = cmake<R>(k == index ? R(1) : R(0), R(0));
  if (bid == 0)
    for (int j = threadIdx.x; j < n_ops; j += kThreads) {
      double th = theta[j], c = 1.0;
      coefs[6 * j] = 1.0;
      for (int m = 1; m <= 5; ++m) {
        c = c * th / (double)m;
        coefs[6 * j + m] = c;
      }
    }
}

// With `mask` set (psi set, n >= 8) also mask = the nonzero octets of
// |index>: the one bit of index's octet; with a chain list as well, the list
// = {index} (its amplitude mask the one bit of index), ready for a forward
// chain.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_setup(C_t<R>* psi, int n, uint64_t index, const double* theta, int n_ops, double* coefs, uint32_t* mask,
        ChainList cl) {
  setup_body<R>(psi, n, index, theta, n_ops, coefs, blockIdx.x, gridDim.x);
  if (mask) {
    const uint32_t words = 1u << (n - 8), iw = (uint32_t)(index >> 8);
    for (uint32_t w = blockIdx.x * kThreads + threadIdx.x; w < words; w += gridDim.x * kThreads)
      mask[w] = w == iw ? 1u << ((index >> 3) & 31u) : 0u;
    if (cl.list) {
      const uint32_t aw = 1u << (n - 5), ia = (uint32_t)(index >> 5);
      for (uint32_t w = blockIdx.x * kThreads + threadIdx.x; w < aw; w += gridDim.x * kThreads)
        cl.amask[w] = w == ia ? 1u << (index & 31u) : 0u;
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the forward chain's step 0 reads slot 2 and appends in slot 0
        cl.list[0] = (uint32_t)index;
        cl.cnt[kRingBase(2)] = 1u;
        cl.cnt[kRingAdd(2)] = 0u;
        cl.cnt[kRingAdd(0)] = 0u;
      }
    }
  }
}

// ------------------------------------------------------------ small kernels

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_norm(const C_t<R>* psi, uint64_t dim, double* partials, unsigned int* counter, double* out) {
  __shared__ double tot[1];
  double v[1] = {0.0};
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < dim;
       k += (uint64_t)gridDim.x * blockDim.x) {
    C_t<R> a = psi[k];
    v[0] += (double)a.x * a.x + (double)a.y * a.y;
  }
  grid_sum<1>(v, partials, counter, gridDim.x, blockIdx.x, out, tot);
}

// lambda = (hpsi - E psi) / <psi|psi> in place over hpsi (E, <psi|psi> = scal[0..1]).
template <typename R>
__device__ void residual_body(const C_t<R>* psi, C_t<R>* hpsi, int n, const double* scal, int bid,
                              int nb) {
  const uint64_t dim = 1ull << n;
  const R er = (R)scal[0], ir = (R)(1.0 / scal[1]);
  for (uint64_t k = bid * (uint64_t)kThreads + threadIdx.x; k < dim; k += (uint64_t)nb * kThreads) {
    C_t<R> h = hpsi[k], p = psi[k];
    hpsi[k] = cmake<R>((h.x - er * p.x) * ir, (h.y - er * p.y) * ir);
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_residual(const C_t<R>* psi, C_t<R>* hpsi, int n, const double* scal) {
  residual_body<R>(psi, hpsi, n, scal, blockIdx.x, gridDim.x);
}

// grads[porder[i]] = 2 raw[i] / <psi|psi>.
__global__ void k_grad_final(const double* raw, const int32_t* porder, int m, const double* scal,
                             double* grads) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) grads[porder[i]] = 2.0 * raw[i] / scal[1];
}

// Largest |g| with a relative tie window; the lowest index among ties wins.
__global__ void k_select(const double* g, int m, double tie_rel, int32_t* out) {
  __shared__ double best[kThreads];
  __shared__ int bidx[kThreads];
  double mx = 0.0;
  for (int i = threadIdx.x; i < m; i += kThreads) mx = fmax(mx, fabs(g[i]));
  best[threadIdx.x] = mx;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) best[threadIdx.x] = fmax(best[threadIdx.x], best[threadIdx.x + s]);
    __syncthreads();
  }
  const double thr = best[0] * (1.0 - tie_rel);
  int idx = m;
  for (int i = threadIdx.x; i < m; i += kThreads)
    if (fabs(g[i]) >= thr && i < idx) idx = i;
  bidx[threadIdx.x] = idx;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) bidx[threadIdx.x] = min(bidx[threadIdx.x], bidx[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = bidx[0] < m ? bidx[0] : -1;
}

// ------------------------------------------------------------ H psi + energy

// H psi layout: a thread owns kAmpsH adjacent amplitudes k0 + i (k0 a
// multiple of kAmpsH), a block a tile of kTileH.  For a group with mask x
// the sources of those outputs are the aligned octet at k0 ^ (x & ~7),
// read with vector loads, output i taking source element i ^ (x & 7).
// Groups are sorted by x & 7 so that this permutation is a compile-time
// register renaming inside each chunk.
constexpr int kTileH = kThreads * kAmpsH;
constexpr int kLutChunkH = 64;       // LUT groups staged per chunk

template <typename R>
__device__ __forceinline__ void load_octet(const C_t<R>* __restrict__ psi, uint32_t base, uint64_t dim,
                                           C_t<R> (&v)[kAmpsH]) {
  if (dim >= kAmpsH) {
    if (sizeof(R) == 4) {
      const float4* p = reinterpret_cast<const float4*>(psi + base);
#pragma unroll
      for (int q = 0; q < kAmpsH / 2; ++q) {
        const float4 f = p[q];
        v[2 * q] = cmake<R>((R)f.x, (R)f.y);
        v[2 * q + 1] = cmake<R>((R)f.z, (R)f.w);
      }
    } else {
#pragma unroll
      for (int q = 0; q < kAmpsH; ++q) v[q] = psi[base + q];
    }
  } else {
#pragma unroll
    for (int q = 0; q < kAmpsH; ++q) v[q] = (base + q < dim) ? psi[base + q] : cmake<R>(0, 0);
  }
}

// LUT groups of one chunk, all with x & 7 == XL.
template <typename R, int XL>
__device__ __forceinline__ void lut_chunk(const HLut<R>* s_l, int cn, uint32_t k0,
                                          const C_t<R>* __restrict__ psi, uint64_t dim,
                                          C_t<R> (&acc)[kAmpsH]) {
  if (k0 >= dim) return;   // a thread past the end of a short state reads nothing
  for (int g = 0; g < cn; ++g) {
    const HLut<R>& L = s_l[g];
    const uint32_t lx = L.x, reg = L.reg;
    const uint32_t code0 = (uint32_t)(__popc(k0 & L.v0) & 1) | ((uint32_t)(__popc(k0 & L.v1) & 1) << 1) |
                           ((uint32_t)(__popc(k0 & L.v2) & 1) << 2) | ((uint32_t)(__popc(k0 & L.z0) & 1) << 3);
    if (reg == 0u) {
      // the code does not vary over the octet: one value for all eight
      const R val = L.lut16[code0];
      if (val == R(0)) continue;
      C_t<R> src[kAmpsH];
      load_octet<R>(psi, k0 ^ (lx & ~7u), dim, src);
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) {
        acc[i].x += val * src[i ^ XL].x;
        acc[i].y += val * src[i ^ XL].y;
      }
    } else {
      R val[kAmpsH];
      bool any = false;
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) {
        val[i] = L.lut16[code0 ^ ((reg >> (4 * i)) & 0xFu)];
        any |= val[i] != R(0);
      }
      if (!any) continue;   // no output of this octet couples to the group
      C_t<R> src[kAmpsH];
      load_octet<R>(psi, k0 ^ (lx & ~7u), dim, src);
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) {
        acc[i].x += val[i] * src[i ^ XL].x;
        acc[i].y += val[i] * src[i ^ XL].y;
      }
    }
  }
}

// Term-list groups of one staged chunk, all with x & 7 == XL.
template <typename R, int XL>
__device__ __forceinline__ void term_chunk(const uint32_t* s_x, const int32_t* s_off,
                                           const int32_t* s_mid, const uint64_t* s_bk, int ng,
                                           const uint32_t* zs, const R* ws, uint32_t k0,
                                           const C_t<R>* __restrict__ psi, uint64_t dim,
                                           C_t<R> (&acc)[kAmpsH]) {
  if (k0 >= dim) return;
  for (int g = 0; g < ng; ++g) {
    const uint32_t x = s_x[g];
    const int tbeg = s_off[g], tmid = s_mid[g], tend = s_off[g + 1];
    const uint64_t bk = s_bk[g];
    if (bk != ~0ull) {
      // real weights, bucket m holding the terms with z & 7 == m: sum each
      // bucket with the signs of k0, then D(k0 + i) = sum_m B_m (-1)^popc(i & m),
      // an 8-point Walsh-Hadamard transform
      R b[kAmpsH];
      int t = tbeg;
#pragma unroll
      for (int m = 0; m < kAmpsH; ++m) {
        b[m] = R(0);
        const int cnt = (int)((bk >> (8 * m)) & 0xFFu);
        for (int c = 0; c < cnt; ++c, ++t) b[m] += (__popc(k0 & zs[t]) & 1) ? -ws[t] : ws[t];
      }
#pragma unroll
      for (int hb = 1; hb < kAmpsH; hb <<= 1)
#pragma unroll
        for (int a = 0; a < kAmpsH; ++a)
          if (!(a & hb)) {
            const R u = b[a], v = b[a | hb];
            b[a] = u + v;
            b[a | hb] = u - v;
          }
      C_t<R> src[kAmpsH];
      load_octet<R>(psi, k0 ^ (x & ~7u), dim, src);
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) {
        acc[i].x += b[i] * src[i ^ XL].x;
        acc[i].y += b[i] * src[i ^ XL].y;
      }
      continue;
    }
    R gr[kAmpsH], gi[kAmpsH], cr[kAmpsH], ci[kAmpsH];
#pragma unroll
    for (int i = 0; i < kAmpsH; ++i) gr[i] = gi[i] = cr[i] = ci[i] = R(0);
    sum_terms8<R>(zs, ws, tbeg, tmid, k0, gr, cr, false);
    if (tend > tmid) sum_terms8<R>(zs, ws, tmid, tend, k0, gi, ci, false);
    C_t<R> src[kAmpsH];
    load_octet<R>(psi, k0 ^ (x & ~7u), dim, src);
#pragma unroll
    for (int i = 0; i < kAmpsH; ++i) {
      const C_t<R> p = src[i ^ XL];
      acc[i].x += gr[i] * p.x - gi[i] * p.y;
      acc[i].y += gr[i] * p.y + gi[i] * p.x;
    }
  }
}

#define GOCP_XL_SWITCH(XLV, CALL) \
  switch (XLV) {                  \
    case 0: CALL(0); break;       \
    case 1: CALL(1); break;       \
    case 2: CALL(2); break;       \
    case 3: CALL(3); break;       \
    case 4: CALL(4); break;       \
    case 5: CALL(5); break;       \
    case 6: CALL(6); break;       \
    default: CALL(7); break;      \
  }

// A block sweeps tiles of kTileH output amplitudes; a thread owns the octet
// k0 .. k0+7.  The off-diagonal groups in LUT form and then the term-list
// groups are staged in shared memory chunk by chunk (a single group too
// large for the stage is read from global memory); the diagonal group (x = 0,
// the identity excluded) comes last, with a compensated sum whose high and
// low parts both enter the FP64 energy.  The identity term
// is added as identity*psi[k].  With `partials` set the item's blocks also
// reduce <psi|psi> -> scal[1] and Re<psi|H' psi> -> scal[2] in FP64, and the
// last block sets scal[0] = E = identity + scal[2] / scal[1].
template <typename R>
__device__ void apply_body(const DevTables& tb, const C_t<R>* __restrict__ psi,
                           C_t<R>* __restrict__ out, double identity, double* partials,
                           unsigned int* counter, double* scal, int bid, int nb) {
  __shared__ uint32_t s_x[kChunkGroups];
  __shared__ int32_t s_off[kChunkGroups + 1];
  __shared__ int32_t s_mid[kChunkGroups];
  __shared__ uint64_t s_bk[kChunkGroups];
  __shared__ uint32_t s_z[kChunkTerms];
  __shared__ R s_w[kChunkTerms];
  __shared__ double tot[2];
  __shared__ HLut<R> s_l[kLutChunkH];
  const R* tw = (const R*)tb.tw;
  const R* dw = (const R*)tb.dw;
  const HLut<R>* hl = (const HLut<R>*)tb.hlut;
  const R idr = (R)identity;
  const uint64_t dim = 1ull << tb.n;
  const uint64_t ntiles = (dim + kTileH - 1) / kTileH;
  double v[2] = {0.0, 0.0};
  for (uint64_t tile = bid; tile < ntiles; tile += nb) {
    const uint32_t k0 = (uint32_t)(tile * kTileH) + threadIdx.x * kAmpsH;
    C_t<R> acc[kAmpsH];
#pragma unroll
    for (int i = 0; i < kAmpsH; ++i) acc[i] = cmake<R>(0, 0);
    // off-diagonal groups in LUT form
    for (int c = 0; c < tb.n_lchunks; ++c) {
      const int g0 = tb.lchunk[c], cn = tb.lchunk[c + 1] - g0;
      __syncthreads();
      {
        // 16-byte vector copy of the chunk's descriptors (no bank conflicts)
        const uint4* src4 = reinterpret_cast<const uint4*>(hl + g0);
        uint4* dst4 = reinterpret_cast<uint4*>(s_l);
        const int words = cn * (int)(sizeof(HLut<R>) / sizeof(uint4));
        for (int w = threadIdx.x; w < words; w += kThreads) dst4[w] = src4[w];
      }
      __syncthreads();
#define GOCP_LUT_CALL(XLV) lut_chunk<R, XLV>(s_l, cn, k0, psi, dim, acc)
      GOCP_XL_SWITCH(tb.lchunk_xl[c], GOCP_LUT_CALL)
#undef GOCP_LUT_CALL
    }
    // off-diagonal groups as term lists
    for (int c = 0; c < tb.n_chunks; ++c) {
      const int g0 = tb.chunk_g[c], g1 = tb.chunk_g[c + 1];
      const int t0 = tb.goff[g0], t1 = tb.goff[g1];
      const bool staged = (t1 - t0) <= kChunkTerms;   // chunks never exceed kChunkGroups
      __syncthreads();
      for (int g = g0 + threadIdx.x; g < g1; g += kThreads) {
        s_x[g - g0] = tb.gx[g];
        s_off[g - g0] = tb.goff[g] - t0;
        s_mid[g - g0] = tb.gmid[g] - t0;
        s_bk[g - g0] = tb.gbk[g];
      }
      if (threadIdx.x == 0) s_off[g1 - g0] = t1 - t0;
      if (staged)
        for (int t = t0 + threadIdx.x; t < t1; t += kThreads) {
          s_z[t - t0] = tb.tz[t];
          s_w[t - t0] = tw[t];
        }
      __syncthreads();
      const uint32_t* zs = staged ? s_z : tb.tz + t0;
      const R* ws = staged ? s_w : tw + t0;
#define GOCP_TERM_CALL(XLV) term_chunk<R, XLV>(s_x, s_off, s_mid, s_bk, g1 - g0, zs, ws, k0, psi, dim, acc)
      GOCP_XL_SWITCH(tb.chunk_xl[c], GOCP_TERM_CALL)
#undef GOCP_TERM_CALL
    }
    // diagonal group, last so that its accumulators are not live above
    R dr[kAmpsH], dc[kAmpsH], di[kAmpsH], dd[kAmpsH];
#pragma unroll
    for (int i = 0; i < kAmpsH; ++i) dr[i] = dc[i] = di[i] = dd[i] = R(0);
    sum_terms8<R>(tb.dz, dw, 0, tb.nd_mid, k0, dr, dc, true);
    sum_terms8<R>(tb.dz, dw, tb.nd_mid, tb.nd, k0, di, dd, false);
    if (k0 < dim) {
      C_t<R> own[kAmpsH];
      load_octet<R>(psi, k0, dim, own);
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) {
        if (k0 + i >= dim) continue;
        const C_t<R> p = own[i];
        const double pp = (double)p.x * p.x + (double)p.y * p.y;
        v[0] += pp;
        // Re(conj(p) (acc + D0 p)); the imaginary diagonal part adds nothing
        v[1] += (double)p.x * acc[i].x + (double)p.y * acc[i].y + ((double)dr[i] - (double)dc[i]) * pp;
        const R d0 = dr[i] - dc[i] + idr;
        out[k0 + i] = cmake<R>(acc[i].x + d0 * p.x - di[i] * p.y, acc[i].y + d0 * p.y + di[i] * p.x);
      }
    }
  }
  if (partials && grid_sum<2>(v, partials, counter, nb, bid, scal + 1, tot)) {
    if (threadIdx.x == 0) scal[0] = identity + tot[1] / tot[0];
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? GOCP_APPLY_MIN_BLOCKS_C64 : 2)
k_apply_h(DevTables tb, const C_t<R>* __restrict__ psi, C_t<R>* __restrict__ out, double identity,
          double* partials, unsigned int* counter, double* scal) {
  apply_body<R>(tb, psi, out, identity, partials, counter, scal, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------ pool strings

// One generator staged for the pair kernels.  D(b) = sum w_t chi_t(b) and
// D(b^x) = sum w2_t chi_t(b), chi_t(b) = (-1)^popc(b & z_t): one parity per
// string gives both ends of a pair.
template <typename R>
struct OpView {
  uint32_t x;
  int nm, ne;            // [0, nm) real weights, [nm, ne) imaginary
  const uint32_t* z;
  const R* w;
  const R* w2;
};

template <typename R>
__device__ __forceinline__ void op_d(const OpView<R>& o, uint32_t b, C_t<R>& d1, C_t<R>& d2) {
  R r1 = 0, r2 = 0, i1 = 0, i2 = 0;
  for (int t = 0; t < o.nm; ++t) {
    const bool odd = __popc(b & o.z[t]) & 1;
    r1 += odd ? -o.w[t] : o.w[t];
    r2 += odd ? -o.w2[t] : o.w2[t];
  }
  for (int t = o.nm; t < o.ne; ++t) {
    const bool odd = __popc(b & o.z[t]) & 1;
    i1 += odd ? -o.w[t] : o.w[t];
    i2 += odd ? -o.w2[t] : o.w2[t];
  }
  d1 = cmake<R>(r1, i1);
  d2 = cmake<R>(r2, i2);
}

// Resolves ops[j] (flagging out-of-range indices: the step then acts as the
// identity) and stages its strings in shared memory when they fit.
template <typename R>
__device__ bool load_op(const DevTables& tb, const int32_t* ops, int j, int32_t* err, int bid,
                        uint32_t* s_z, R* s_w, R* s_w2, OpView<R>& o) {
  const int op = ops[j];
  if (op < 0 || op >= tb.M) {
    if (bid == 0 && threadIdx.x == 0) atomicOr(err, 1);
    return false;
  }
  const int sb = tb.poff[op], sm = tb.pmid[op], se = tb.poff[op + 1];
  const R* pw = (const R*)tb.pw;
  const R* pw2 = (const R*)tb.pw2;
  o.x = tb.px[op];
  o.nm = sm - sb;
  o.ne = se - sb;
  if (se - sb <= kStageStrings) {
    for (int t = threadIdx.x; t < se - sb; t += blockDim.x) {
      s_z[t] = tb.pz[sb + t];
      s_w[t] = pw[sb + t];
      s_w2[t] = pw2[sb + t];
    }
    __syncthreads();
    o.z = s_z;
    o.w = s_w;
    o.w2 = s_w2;
  } else {
    o.z = tb.pz + sb;
    o.w = pw + sb;
    o.w2 = pw2 + sb;
  }
  return true;
}

__device__ __forceinline__ uint32_t pair_base(uint64_t p, int s) {
  // insert a 0 at bit s of p
  return (uint32_t)(((p >> s) << (s + 1)) | (p & ((1ull << s) - 1)));
}

// Compensated complex accumulation (FP32 path); plain for FP64.
template <typename R>
__device__ __forceinline__ void kahan_add(C_t<R>& s, C_t<R>& c, C_t<R> v) {
  if (sizeof(R) == 4) {
    R yx = v.x - c.x, yy = v.y - c.y;
    R tx = s.x + yx, ty = s.y + yy;
    c.x = (tx - s.x) - yx;
    c.y = (ty - s.y) - yy;
    s.x = tx;
    s.y = ty;
  } else {
    s.x += v.x;
    s.y += v.y;
  }
}

// ------------------------------------------------------------ Taylor step

// psi <- T(theta_j A_{ops[j]}) psi: on each pair (b, b^x) the chain
// v_m = A v_{m-1} (Eq. 6) and the partial sum of Eq. (5), taken in order
// m = 0..5, stay in registers.
// Chain lists (ChainList): membership, append, and the end of a step.
__device__ __forceinline__ bool chain_listed(const ChainList& cl, uint32_t k) {
  return (cl.amask[k >> 5] >> (k & 31u)) & 1u;
}

// k (not listed, its amplitude now nonzero) joins the list at base + the
// step's count (ring slot cur); its octet's bit is set in mask as well.  Past
// cap the index is not stored (the list is then incomplete and later steps
// enumerate pairs).
__device__ __forceinline__ void chain_append(const ChainList& cl, uint32_t k, uint32_t base, int cur,
                                             uint32_t* mask) {
  const uint32_t bit = 1u << (k & 31u);
  if (atomicOr(cl.amask + (k >> 5), bit) & bit) return;
  const uint32_t pos = base + atomicAdd(cl.cnt + kRingAdd(cur), 1u);
  if (pos < cl.cap) cl.list[pos] = k;
  octet_set(mask, k);
}


// Start of step j of a chain (forward: the previous step was j - 1, the
// next is j + 1; reverse: j + 1 and j - 1): the list length at the start
// (read once per block), recorded in this step's slot by block 0, and the
// next step's counter cleared.  Called by every thread of the block.
__device__ __forceinline__ uint32_t chain_begin(const ChainList& cl, int j, bool forward, int* cur) {
  __shared__ uint32_t s_n0;
  const int prev = (j + (forward ? 2 : 1)) % 3, next = (j + (forward ? 1 : 2)) % 3;
  *cur = j % 3;
  if (threadIdx.x == 0) {
    s_n0 = cl.cnt[kRingBase(prev)] + cl.cnt[kRingAdd(prev)];
    if (blockIdx.x == 0) {
      cl.cnt[kRingBase(*cur)] = s_n0;
      cl.cnt[kRingAdd(next)] = 0u;
    }
  }
  __syncthreads();
  return s_n0;
}

// LUT form of the same step: real D on the pair; only the pairs the
// operator touches are visited (enumerated, see PairEnum) -- on the others
// T = I and nothing is read or written.
// With `mask` set (a nonzero-octet mask of psi, see octet_bit) a pair whose
// two octets are marked zero is skipped -- T maps (0, 0) to (0, 0) -- and a
// pair that is computed marks both of its octets, so that the mask stays
// valid for the updated psi.
// With `mask` and a complete chain list (tb.cl), the step walks the listed
// nonzero amplitudes instead of the operator's pairs: a touched pair is
// computed once, by its base's entry if the base is listed, else by its
// partner's; a pair with neither end listed is zero and stays zero; the
// unlisted end of a computed pair joins the list when it becomes nonzero.
// p1, p2: the amplitudes of b and b ^ x (wherever they are held).
template <typename R>
__device__ __forceinline__ void taylor_pair_at(const LutDev<R>& L, const R (&c)[6], uint32_t b, uint32_t ph,
                                               C_t<R>* p1, C_t<R>* p2, C_t<R>& o1, C_t<R>& o2) {
  const uint32_t phx = L.fx & 7u, sgx = (L.fx >> 3) & 1u;
  const R l1 = L.lut[ph], l2 = L.lut[ph ^ phx];
  const uint32_t sg = __popc(b & L.z0) & 1u;
  const R d1 = sg ? -l1 : l1, d2 = (sg ^ sgx) ? -l2 : l2;
  const C_t<R> v1 = *p1, v2 = *p2;
  if constexpr (sizeof(R) == 8) {
    // complex128: the same fifth-order polynomial evaluated through
    // A^2 = mu I on the pair (mu = D1 D2): T = C I + S A with
    // C = c0 + c2 mu + c4 mu^2, S = c1 + c3 mu + c5 mu^2 -- 16 FP64
    // operations instead of the chain's 40, on a pipe about 1/64 the width
    // of FP32 here
    const R mu = d1 * d2, mu2 = mu * mu;
    const R cc = c[0] + c[2] * mu + c[4] * mu2;
    const R sc = c[1] + c[3] * mu + c[5] * mu2;
    const R sd1 = sc * d1, sd2 = sc * d2;
    o1 = cmake<R>(cc * v1.x + sd1 * v2.x, cc * v1.y + sd1 * v2.y);
    o2 = cmake<R>(cc * v2.x + sd2 * v1.x, cc * v2.y + sd2 * v1.y);
  } else {
    // complex64: the literal chain v_m = A v_(m-1) with compensated sums
    C_t<R> w1 = v1, w2 = v2;
    C_t<R> s1 = v1, s2 = v2, e1 = cmake<R>(0, 0), e2 = cmake<R>(0, 0);
#pragma unroll
    for (int m = 1; m <= 5; ++m) {
      C_t<R> n1 = cscale<R>(w2, d1), n2 = cscale<R>(w1, d2);   // (A v)[b] = D(b) v[b^x]
      w1 = n1;
      w2 = n2;
      kahan_add<R>(s1, e1, cscale<R>(w1, c[m]));
      kahan_add<R>(s2, e2, cscale<R>(w2, c[m]));
    }
    o1 = csub<R>(s1, e1);
    o2 = csub<R>(s2, e2);
  }
  *p1 = o1;
  *p2 = o2;
}

template <typename R>
__device__ __forceinline__ void taylor_pair(const LutDev<R>& L, const R (&c)[6], uint32_t b, uint32_t ph, C_t<R>* psi,
                                            C_t<R>& o1, C_t<R>& o2) {
  taylor_pair_at<R>(L, c, b, ph, psi + b, psi + (b ^ L.x), o1, o2);
}

template <typename R>
__device__ void taylor_lut_body(const DevTables& tb, const int32_t* ops, const double* coefs, int j,
                                C_t<R>* psi, int32_t* err, int bid, int nb, uint32_t* mask) {
  const int op = ops[j];
  if (op < 0 || op >= tb.M) {
    if (bid == 0 && threadIdx.x == 0) atomicOr(err, 1);
    return;
  }
  const LutDev<R>& L = ((const LutDev<R>*)tb.plut)[op];   // read in place: L.lut is indexed at run time
  const PairEnum& E = tb.penum[op];
  R c[6];
  step_coefs<R>(coefs, j, c);
  const uint32_t phx = L.fx & 7u;
  const ChainList& cl = tb.cl;
  if (mask && cl.list) {
    int cur;
    const uint32_t n0 = chain_begin(cl, j, true, &cur);
    if (n0 <= cl.cap) {
      for (uint32_t q = bid * kThreads + threadIdx.x; q < n0; q += (uint32_t)nb * kThreads) {
        const uint32_t k = cl.list[q];
        // the pair's base; untouched pairs (T = I) are passed over before
        // the membership read, which only a touched pair needs
        const uint32_t b = ((k >> L.s) & 1u) ? k ^ L.x : k;
        const uint32_t ph = lut_phi(L, b);
        if (rzero<R>(L.lut[ph]) && rzero<R>(L.lut[ph ^ phx])) continue;   // T = I on the pair
        if (b != k && chain_listed(cl, b)) continue;   // the base's entry computes the pair
        C_t<R> o1, o2;
        taylor_pair<R>(L, c, b, ph, psi, o1, o2);
        const uint32_t other = b == k ? b ^ L.x : b;
        const C_t<R> ov = b == k ? o2 : o1;
        if (!(rzero<R>(ov.x) && rzero<R>(ov.y)) && !chain_listed(cl, other)) chain_append(cl, other, n0, cur, mask);
      }
      return;
    }
  }
  const uint64_t count = (uint64_t)E.ncodes << E.log2cnt;
  for (uint64_t q = bid * (uint64_t)kThreads + threadIdx.x; q < count; q += (uint64_t)nb * kThreads) {
    uint32_t ph;
    const uint32_t b = enum_pair(E, (uint32_t)q, &ph);
    const uint32_t b2 = b ^ L.x;
    uint32_t m1 = 1u, m2 = 1u;
    if (mask) {
      m1 = octet_bit(mask, b);
      m2 = octet_bit(mask, b2);
      if (!(m1 | m2)) continue;
    }
    C_t<R> o1, o2;
    taylor_pair<R>(L, c, b, ph, psi, o1, o2);
    if (!m1) octet_set(mask, b);
    if (!m2) octet_set(mask, b2);
  }
}

// `mask` is used (and kept valid) by the LUT form only; the generic form
// neither reads nor updates it, so callers pass it only for LUT pools.
template <typename R>
__device__ void taylor_body(const DevTables& tb, const int32_t* ops, const double* coefs, int j,
                            C_t<R>* psi, int32_t* err, int bid, int nb, uint32_t* mask = nullptr) {
  if (tb.pool_lut) {
    taylor_lut_body<R>(tb, ops, coefs, j, psi, err, bid, nb, mask);
    return;
  }
  __shared__ uint32_t s_z[kStageStrings];
  __shared__ R s_w[kStageStrings], s_w2[kStageStrings];
  OpView<R> o;
  if (!load_op<R>(tb, ops, j, err, bid, s_z, s_w, s_w2, o)) return;
  R c[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) c[m] = (R)coefs[6 * j + m];
  const int s = __ffs(o.x) - 1;
  const uint64_t npairs = 1ull << (tb.n - 1);
  for (uint64_t p = bid * (uint64_t)kThreads + threadIdx.x; p < npairs; p += (uint64_t)nb * kThreads) {
    const uint32_t b = pair_base(p, s), b2 = b ^ o.x;
    C_t<R> d1, d2;
    op_d<R>(o, b, d1, d2);
    C_t<R> v1 = psi[b], v2 = psi[b2];
    C_t<R> s1 = v1, s2 = v2, e1 = cmake<R>(0, 0), e2 = cmake<R>(0, 0);
#pragma unroll
    for (int m = 1; m <= 5; ++m) {
      C_t<R> n1 = cmul<R>(d1, v2), n2 = cmul<R>(d2, v1);   // (A v)[b] = D(b) v[b^x]
      v1 = n1;
      v2 = n2;
      kahan_add<R>(s1, e1, cscale<R>(v1, c[m]));
      kahan_add<R>(s2, e2, cscale<R>(v2, c[m]));
    }
    psi[b] = csub<R>(s1, e1);
    psi[b2] = csub<R>(s2, e2);
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_taylor5(DevTables tb, const int32_t* ops, const double* coefs, int j, C_t<R>* psi, int32_t* err,
          uint32_t* mask) {
  chain_step_begin();
  taylor_body<R>(tb, ops, coefs, j, psi, err, blockIdx.x, gridDim.x, mask);
}

// ------------------------------------------------------------ adjoint step

// Backward step j of the adjoint sweep.  On each pair A = [[0, D1], [D2, 0]],
// A^2 = mu I with mu = D1 D2, so T = C I + S A with C = c0 + c2 mu + c4 mu^2,
// S = c1 + c3 mu + c5 mu^2 (c_m = theta^m/m!), and T' = dT/dtheta =
// C' I + S' A with C' = c1 mu + c3 mu^2, S' = C.  In place:
//   psi <- T^-1 psi = (C I - S A) psi / (C^2 - S^2 mu)      (exact inverse)
//   dE_j += 2 Re <lambda|T' psi>                            (lambda before update)
//   lambda <- T^dagger lambda.
// LUT form of the backward step (real D) over the enumerated pairs the
// operator touches (elsewhere T = I and T' = 0).
// With `mask` set (nonzero octets of psi or lambda) a pair on which both are
// zero is skipped -- it adds nothing to dE and stays zero -- and a computed
// pair marks both of its octets.
// p1, p2 / q1, q2: the psi / lambda amplitudes of b and b ^ x.
template <typename R>
__device__ __forceinline__ double adjoint_pair_at(const LutDev<R>& L, const R (&c)[6], uint32_t b, uint32_t ph,
                                                  C_t<R>* p1, C_t<R>* p2, C_t<R>* q1p, C_t<R>* q2p,
                                                  C_t<R> (&out)[4]) {
  const uint32_t phx = L.fx & 7u, sgx = (L.fx >> 3) & 1u;
  const R l1 = L.lut[ph], l2 = L.lut[ph ^ phx];
  const uint32_t sg = __popc(b & L.z0) & 1u;
  const R d1 = sg ? -l1 : l1, d2 = (sg ^ sgx) ? -l2 : l2;
  const R mu = d1 * d2, mu2 = mu * mu;
  const R cc = c[0] + c[2] * mu + c[4] * mu2;
  const R sc = c[1] + c[3] * mu + c[5] * mu2;
  const R cd = c[1] * mu + c[3] * mu2;
  const R inv = R(1) / (cc * cc - sc * sc * mu);
  const R sd1 = sc * d1, sd2 = sc * d2;
  const C_t<R> u1 = *p1, u2 = *p2;
  const C_t<R> q1 = cscale<R>(csub<R>(cscale<R>(u1, cc), cscale<R>(u2, sd1)), inv);
  const C_t<R> q2 = cscale<R>(csub<R>(cscale<R>(u2, cc), cscale<R>(u1, sd2)), inv);
  const C_t<R> t1 = cadd<R>(cscale<R>(q1, cd), cscale<R>(q2, cc * d1));
  const C_t<R> t2 = cadd<R>(cscale<R>(q2, cd), cscale<R>(q1, cc * d2));
  const C_t<R> l1v = *q1p, l2v = *q2p;
  // the pair's term of 2 Re<lambda|T' psi>, formed in R (one conversion)
  const double v = 2.0 * (double)(l1v.x * t1.x + l1v.y * t1.y + l2v.x * t2.x + l2v.y * t2.y);
  out[0] = q1;
  out[1] = q2;
  out[2] = cadd<R>(cscale<R>(l1v, cc), cscale<R>(l2v, sd2));
  out[3] = cadd<R>(cscale<R>(l1v, sd1), cscale<R>(l2v, cc));
  *p1 = out[0];
  *p2 = out[1];
  *q1p = out[2];
  *q2p = out[3];
  return v;
}

template <typename R>
__device__ __forceinline__ double adjoint_pair(const LutDev<R>& L, const R (&c)[6], uint32_t b, uint32_t ph,
                                               C_t<R>* psi, C_t<R>* lam, C_t<R> (&out)[4]) {
  const uint32_t b2 = b ^ L.x;
  return adjoint_pair_at<R>(L, c, b, ph, psi + b, psi + b2, lam + b, lam + b2, out);
}

// dpart set: each block writes its partial of dE_j to dpart[j nb + bid]
// (k_dtheta_reduce adds them after the sweep) instead of the in-step grid
// reduction into dtheta[j].
template <typename R>
__device__ void adjoint_lut_body(const DevTables& tb, const int32_t* ops, const double* coefs, int j,
                                 C_t<R>* psi, C_t<R>* lam, double* partials, unsigned int* counter,
                                 double* dtheta, int32_t* err, int bid, int nb, uint32_t* mask, double* dpart) {
  __shared__ double tot[1];
  __shared__ double s_red[kWarps];
  const int op = ops[j];
  if (op < 0 || op >= tb.M) {
    if (bid == 0 && threadIdx.x == 0) {
      atomicOr(err, 1);
      dtheta[j] = 0.0;
    }
    if (dpart && threadIdx.x == 0) dpart[(size_t)j * nb + bid] = 0.0;
    return;
  }
  const LutDev<R>& L = ((const LutDev<R>*)tb.plut)[op];   // read in place: L.lut is indexed at run time
  const PairEnum& E = tb.penum[op];
  R c[6];
  step_coefs<R>(coefs, j, c);
  const uint32_t phx = L.fx & 7u;
  double v[1] = {0.0};
  const ChainList& cl = tb.cl;
  int cur = 0;
  const uint32_t n0 = mask && cl.list ? chain_begin(cl, j, false, &cur) : 0xFFFFFFFFu;
  if (n0 <= cl.cap) {
    // the listed amplitudes, nonzero in psi or lambda (see taylor_lut_body)
    for (uint32_t q = bid * kThreads + threadIdx.x; q < n0; q += (uint32_t)nb * kThreads) {
      const uint32_t k = cl.list[q];
      const uint32_t b = ((k >> L.s) & 1u) ? k ^ L.x : k;   // the pair's base
      const uint32_t ph = lut_phi(L, b);
      if (rzero<R>(L.lut[ph]) && rzero<R>(L.lut[ph ^ phx])) continue;   // T = I, T' = 0 on the pair
      if (b != k && chain_listed(cl, b)) continue;   // the base's entry computes the pair
      C_t<R> o[4];
      v[0] += adjoint_pair<R>(L, c, b, ph, psi, lam, o);
      const bool base = b == k;
      const uint32_t other = base ? b ^ L.x : b;
      const C_t<R> op1 = base ? o[1] : o[0], ol1 = base ? o[3] : o[2];
      if (!(rzero<R>(op1.x) && rzero<R>(op1.y) && rzero<R>(ol1.x) && rzero<R>(ol1.y)) && !chain_listed(cl, other))
        chain_append(cl, other, n0, cur, mask);
    }
  } else {
    const uint64_t count = (uint64_t)E.ncodes << E.log2cnt;
    for (uint64_t q = bid * (uint64_t)kThreads + threadIdx.x; q < count; q += (uint64_t)nb * kThreads) {
      uint32_t ph;
      const uint32_t b = enum_pair(E, (uint32_t)q, &ph);
      const uint32_t b2 = b ^ L.x;
      uint32_t m1 = 1u, m2 = 1u;
      if (mask) {
        m1 = octet_bit(mask, b);
        m2 = octet_bit(mask, b2);
        if (!(m1 | m2)) continue;
      }
      C_t<R> o[4];
      v[0] += adjoint_pair<R>(L, c, b, ph, psi, lam, o);
      if (!m1) octet_set(mask, b);
      if (!m2) octet_set(mask, b2);
    }
  }
  if (!dpart) {
    grid_sum<1>(v, partials, counter, nb, bid, dtheta + j, tot);
    return;
  }
  // most warps touched no pair: their FP64 reduction is skipped
  const double w = __any_sync(0xffffffffu, v[0] != 0.0) ? warp_sum(v[0]) : 0.0;
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kWarps; ++q) t += s_red[q];
    dpart[(size_t)j * nb + bid] = t;
  }
}

// dtheta[j] = sum_b dpart[j nb + b], j < n_ops (one block per j).
__global__ void __launch_bounds__(kThreads) k_dtheta_reduce(const double* dpart, int nb, double* dtheta) {
  __shared__ double s_red[kWarps];
  const int j = blockIdx.x;
  double t = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) t += dpart[(size_t)j * nb + b];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int q = 0; q < kWarps; ++q) u += s_red[q];
    dtheta[j] = u;
  }
}

template <typename R>
__device__ void adjoint_body(const DevTables& tb, const int32_t* ops, const double* coefs, int j,
                             C_t<R>* psi, C_t<R>* lam, double* partials, unsigned int* counter,
                             double* dtheta, int32_t* err, int bid, int nb, uint32_t* mask = nullptr,
                             double* dpart = nullptr) {
  if (tb.pool_lut) {
    adjoint_lut_body<R>(tb, ops, coefs, j, psi, lam, partials, counter, dtheta, err, bid, nb, mask, dpart);
    return;
  }
  __shared__ uint32_t s_z[kStageStrings];
  __shared__ R s_w[kStageStrings], s_w2[kStageStrings];
  __shared__ double tot[1];
  OpView<R> o;
  if (!load_op<R>(tb, ops, j, err, bid, s_z, s_w, s_w2, o)) {
    if (bid == 0 && threadIdx.x == 0) dtheta[j] = 0.0;
    return;
  }
  R c[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) c[m] = (R)coefs[6 * j + m];
  const int s = __ffs(o.x) - 1;
  const uint64_t npairs = 1ull << (tb.n - 1);
  double v[1] = {0.0};
  for (uint64_t p = bid * (uint64_t)kThreads + threadIdx.x; p < npairs; p += (uint64_t)nb * kThreads) {
    const uint32_t b = pair_base(p, s), b2 = b ^ o.x;
    C_t<R> d1, d2;
    op_d<R>(o, b, d1, d2);
    const C_t<R> mu = cmul<R>(d1, d2), mu2 = cmul<R>(mu, mu);
    const C_t<R> cc = cmake<R>(c[0] + c[2] * mu.x + c[4] * mu2.x, c[2] * mu.y + c[4] * mu2.y);
    const C_t<R> sc = cmake<R>(c[1] + c[3] * mu.x + c[5] * mu2.x, c[3] * mu.y + c[5] * mu2.y);
    const C_t<R> cd = cmake<R>(c[1] * mu.x + c[3] * mu2.x, c[1] * mu.y + c[3] * mu2.y);
    const C_t<R> det = csub<R>(cmul<R>(cc, cc), cmul<R>(cmul<R>(sc, sc), mu));
    const R dn = det.x * det.x + det.y * det.y;
    const C_t<R> inv = cmake<R>(det.x / dn, -det.y / dn);
    const C_t<R> sd1 = cmul<R>(sc, d1), sd2 = cmul<R>(sc, d2);
    const C_t<R> u1 = psi[b], u2 = psi[b2];
    const C_t<R> q1 = cmul<R>(csub<R>(cmul<R>(cc, u1), cmul<R>(sd1, u2)), inv);
    const C_t<R> q2 = cmul<R>(csub<R>(cmul<R>(cc, u2), cmul<R>(sd2, u1)), inv);
    const C_t<R> t1 = cadd<R>(cmul<R>(cd, q1), cmul<R>(cmul<R>(cc, d1), q2));
    const C_t<R> t2 = cadd<R>(cmul<R>(cd, q2), cmul<R>(cmul<R>(cc, d2), q1));
    const C_t<R> l1 = lam[b], l2 = lam[b2];
    v[0] += 2.0 * ((double)l1.x * t1.x + (double)l1.y * t1.y + (double)l2.x * t2.x +
                   (double)l2.y * t2.y);
    psi[b] = q1;
    psi[b2] = q2;
    lam[b] = cadd<R>(cmul<R>(cconj<R>(cc), l1), cmul<R>(cconj<R>(sd2), l2));
    lam[b2] = cadd<R>(cmul<R>(cconj<R>(sd1), l1), cmul<R>(cconj<R>(cc), l2));
  }
  grid_sum<1>(v, partials, counter, nb, bid, dtheta + j, tot);
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_adjoint(DevTables tb, const int32_t* ops, const double* coefs, int j, C_t<R>* psi, C_t<R>* lam,
          double* partials, unsigned int* counter, double* dtheta, int32_t* err, uint32_t* mask, double* dpart) {
  chain_step_begin();
  adjoint_body<R>(tb, ops, coefs, j, psi, lam, partials, counter, dtheta, err, blockIdx.x, gridDim.x, mask,
                  dpart);
}

// ------------------------------------------------------------ on-chip chains
//
// A state that fits one block's shared memory (kSmemStateBytes: 2^14
// complex64 or 2^13 complex128 amplitudes for the forward chain; the
// backward sweep holds psi and lambda, so 2^13 / 2^12) runs its whole chain
// in one launch: the block loads the state, applies every step of the
// ansatz in order with a barrier between steps, and stores it back.  Each
// step visits the operator's enumerated touched pairs with the same per-pair
// arithmetic as the one-launch-per-step kernels (taylor_pair, adjoint_pair),
// so the forward chain gives the same state bit for bit; the backward sweep
// sums each dE_j over the block in a fixed order.  A step costs one pass of
// the block over shared memory instead of a grid launch.
constexpr int kSmemThreads = 1024;
constexpr uint32_t kSmemStateBytes = 128u << 10;
constexpr uint32_t kSmemDescBytes = 16u << 10;   // staged step descriptors (kStepChunk StepDesc)

template <typename R>
__device__ __forceinline__ void smem_copy_in(C_t<R>* dst, const C_t<R>* src, uint32_t dim) {
  const uint32_t n16 = dim * (uint32_t)sizeof(C_t<R>) / 16u;
  for (uint32_t i = threadIdx.x; i < n16; i += kSmemThreads)
    reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
}

template <typename R>
__device__ __forceinline__ void smem_copy_out(C_t<R>* dst, const C_t<R>* src, uint32_t dim) {
  const uint32_t n16 = dim * (uint32_t)sizeof(C_t<R>) / 16u;
  for (uint32_t i = threadIdx.x; i < n16; i += kSmemThreads)
    reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
}

template <typename R>
__device__ __forceinline__ bool cz(const C_t<R>& v) { return v.x == R(0) && v.y == R(0); }

// One step's operator, staged in shared memory ahead of the steps that use
// it, so that a step reads no descriptor from global memory.
template <typename R>
struct StepDesc {
  LutDev<R> L;
  PairEnum E;
  R c[6];     // theta^m / m!, m = 0..5
  int valid;  // 0: the operator index was out of range (the step is the identity)
};
constexpr int kStepChunk = 64;   // steps staged at a time
static_assert(kStepChunk * sizeof(StepDesc<double>) <= (16u << 10), "staged steps fit kSmemDescBytes");

template <typename T>
__device__ __forceinline__ void copy_words(T* dst, const T* src) {
  static_assert(sizeof(T) % 4 == 0, "word copy");
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int w = (int)(threadIdx.x & 31); w < (int)(sizeof(T) / 4); w += 32) d[w] = s[w];
}

// sd[i] = step j0 + i for i < j1 - j0 (one warp per step); flags an
// out-of-range operator in err when `flag`.  Ends with a block barrier.
template <typename R>
__device__ void stage_steps(const DevTables& tb, const int32_t* ops, const double* coefs, int j0, int j1,
                            StepDesc<R>* sd, int32_t* err, bool flag) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < j1 - j0; i += kSmemThreads / 32) {
    const int j = j0 + i, op = ops[j];
    const bool ok = op >= 0 && op < tb.M;
    if (lane == 0) sd[i].valid = ok ? 1 : 0;
    if (!ok) {
      if (flag && lane == 0) atomicOr(err, 1);
      continue;
    }
    copy_words(&sd[i].L, ((const LutDev<R>*)tb.plut) + op);
    copy_words(&sd[i].E, tb.penum + op);
    if (lane < 6) sd[i].c[lane] = (R)coefs[6 * j + lane];
  }
  __syncthreads();
}

// psi <- T(theta_{P-1} A_{ops[P-1]}) ... T(theta_0 A_{ops[0]}) psi, LUT pools
// only, by one block of kSmemThreads threads with the state in sp (shared
// memory).  With mask set, also writes the exact nonzero-octet mask of the
// result (see octet_mask).
template <typename R>
__device__ void taylor_chain_smem_body(const DevTables& tb, const int32_t* ops, const double* coefs, int n_ops,
                                       C_t<R>* psi, int32_t* err, uint32_t* mask, C_t<R>* sp) {
  const uint32_t dim = 1u << tb.n;
  StepDesc<R>* sd = reinterpret_cast<StepDesc<R>*>(sp + dim);
  smem_copy_in<R>(sp, psi, dim);
  for (int j = 0; j < n_ops; ++j) {
    if (j % kStepChunk == 0) stage_steps<R>(tb, ops, coefs, j, min(n_ops, j + kStepChunk), sd, err, true);
    const StepDesc<R>& D = sd[j % kStepChunk];
    if (!D.valid) continue;   // acts as the identity, flagged
    const LutDev<R>& L = D.L;
    const PairEnum& E = D.E;
    R c[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) c[m] = D.c[m];
    const uint32_t count = (uint32_t)E.ncodes << E.log2cnt;
    for (uint32_t q = threadIdx.x; q < count; q += kSmemThreads) {
      uint32_t ph;
      const uint32_t b = enum_pair(E, q, &ph);
      if (cz<R>(sp[b]) && cz<R>(sp[b ^ L.x])) continue;   // T maps (0, 0) to (0, 0)
      C_t<R> o1, o2;
      taylor_pair<R>(L, c, b, ph, sp, o1, o2);
    }
    __syncthreads();
  }
  smem_copy_out<R>(psi, sp, dim);
  if (mask) {
    // one octet per thread; a warp's 32 octets make one mask word
    for (uint32_t o0 = 0; o0 < ((dim + 7u) >> 3); o0 += kSmemThreads) {
      const uint32_t o = o0 + threadIdx.x;
      bool nz = false;
      if (o < (dim >> 3))
        for (int i = 0; i < 8; ++i) nz |= sp[8u * o + i].x != R(0) || sp[8u * o + i].y != R(0);
      const uint32_t word = __ballot_sync(0xffffffffu, nz);
      if ((threadIdx.x & 31) == 0 && o < (dim >> 3)) mask[o >> 5] = word;
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kSmemThreads, 1)
k_taylor_chain_smem(DevTables tb, const int32_t* ops, const double* coefs, int n_ops, C_t<R>* psi,
                    int32_t* err, uint32_t* mask) {
  extern __shared__ __align__(16) uint8_t cs_raw[];
  taylor_chain_smem_body<R>(tb, ops, coefs, n_ops, psi, err, mask, reinterpret_cast<C_t<R>*>(cs_raw));
}

// The backward sweep of the adjoint (see adjoint_pair) for j = P-1 .. 0 over
// psi and lambda, by one block with both in shared memory (sp: 2 states);
// dtheta[j] = the block's fixed-order sum.
template <typename R>
__device__ void adjoint_chain_smem_body(const DevTables& tb, const int32_t* ops, const double* coefs, int n_ops,
                                        C_t<R>* psi, C_t<R>* lam, double* dtheta, int32_t* err, C_t<R>* sp) {
  __shared__ double s_red[kSmemThreads / 32];
  const uint32_t dim = 1u << tb.n;
  C_t<R>* sl = sp + dim;
  StepDesc<R>* sd = reinterpret_cast<StepDesc<R>*>(sl + dim);
  smem_copy_in<R>(sp, psi, dim);
  smem_copy_in<R>(sl, lam, dim);
  for (int j = n_ops - 1; j >= 0; --j) {
    const int jc = j - j % kStepChunk;   // first step of j's chunk
    if (j == n_ops - 1 || j % kStepChunk == kStepChunk - 1)
      stage_steps<R>(tb, ops, coefs, jc, min(n_ops, jc + kStepChunk), sd, err, true);
    const StepDesc<R>& D = sd[j - jc];
    if (!D.valid) {
      if (threadIdx.x == 0) dtheta[j] = 0.0;
      continue;
    }
    const LutDev<R>& L = D.L;
    const PairEnum& E = D.E;
    R c[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) c[m] = D.c[m];
    const uint32_t count = (uint32_t)E.ncodes << E.log2cnt;
    double v = 0.0;
    for (uint32_t q = threadIdx.x; q < count; q += kSmemThreads) {
      uint32_t ph;
      const uint32_t b = enum_pair(E, q, &ph), b2 = b ^ L.x;
      // psi and lambda zero at both ends: nothing to add, and they stay zero
      if (cz<R>(sp[b]) && cz<R>(sp[b2]) && cz<R>(sl[b]) && cz<R>(sl[b2])) continue;
      C_t<R> o[4];
      v += adjoint_pair<R>(L, c, b, ph, sp, sl, o);
    }
    const double w = __any_sync(0xffffffffu, v != 0.0) ? warp_sum(v) : 0.0;
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < kSmemThreads / 32; ++q) t += s_red[q];
      dtheta[j] = t;
    }
    __syncthreads();
  }
  smem_copy_out<R>(psi, sp, dim);
  smem_copy_out<R>(lam, sl, dim);
}

template <typename R>
__global__ void __launch_bounds__(kSmemThreads, 1)
k_adjoint_chain_smem(DevTables tb, const int32_t* ops, const double* coefs, int n_ops, C_t<R>* psi,
                     C_t<R>* lam, double* dtheta, int32_t* err) {
  extern __shared__ __align__(16) uint8_t cs_raw[];
  adjoint_chain_smem_body<R>(tb, ops, coefs, n_ops, psi, lam, dtheta, err, reinterpret_cast<C_t<R>*>(cs_raw));
}

// ------------------------------------------------------------ pool gradients

// blockIdx.y selects kOpsPerBlock operators in GOCP family order; the
// x-slice of blocks sweeps all amplitudes.  raw[i] = Re<H psi|A psi> of the
// i-th operator in family order.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_pool_grad(DevTables tb, const C_t<R>* __restrict__ psi, const C_t<R>* __restrict__ hpsi,
            double* partials, unsigned int* counters, double* raw) {
  __shared__ uint32_t s_x[kOpsPerBlock];
  __shared__ int s_beg[kOpsPerBlock + 1], s_mid[kOpsPerBlock];
  __shared__ uint32_t s_z[kStageStrings];
  __shared__ R s_w[kStageStrings];
  __shared__ int s_glob[kOpsPerBlock];   // op index when its strings are not staged
  __shared__ double tot[kOpsPerBlock];
  const int first = blockIdx.y * kOpsPerBlock;
  const int nops = min(kOpsPerBlock, tb.M - first);
  const R* pw = (const R*)tb.pw;
  if (threadIdx.x == 0) {
    int fill = 0;
    for (int i = 0; i < nops; ++i) {
      const int op = tb.porder[first + i];
      const int sb = tb.poff[op], se = tb.poff[op + 1];
      s_x[i] = tb.px[op];
      s_beg[i] = fill;
      if (fill + (se - sb) <= kStageStrings) {
        s_mid[i] = fill + tb.pmid[op] - sb;
        s_glob[i] = -1;
        fill += se - sb;
      } else {
        s_mid[i] = fill;
        s_glob[i] = op;
      }
      s_beg[i + 1] = fill;
    }
  }
  __syncthreads();
  for (int i = 0; i < nops; ++i) {
    const int op = tb.porder[first + i];
    if (s_glob[i] >= 0) continue;
    const int sb = tb.poff[op], cnt = s_beg[i + 1] - s_beg[i];
    for (int t = threadIdx.x; t < cnt; t += kThreads) {
      s_z[s_beg[i] + t] = tb.pz[sb + t];
      s_w[s_beg[i] + t] = pw[sb + t];
    }
  }
  __syncthreads();
  R acc[kOpsPerBlock], cmp[kOpsPerBlock];
#pragma unroll
  for (int i = 0; i < kOpsPerBlock; ++i) {
    acc[i] = R(0);
    cmp[i] = R(0);
  }
  const uint64_t dim = 1ull << tb.n;
  for (uint64_t kk = blockIdx.x * (uint64_t)kThreads + threadIdx.x; kk < dim;
       kk += (uint64_t)gridDim.x * kThreads) {
    const uint32_t k = (uint32_t)kk;
    const C_t<R> h = hpsi[k];
#pragma unroll
    for (int i = 0; i < kOpsPerBlock; ++i) {
      if (i >= nops) break;
      R dr = 0, di = 0;
      if (s_glob[i] < 0) {
        for (int t = s_beg[i]; t < s_mid[i]; ++t) dr += (__popc(k & s_z[t]) & 1) ? -s_w[t] : s_w[t];
        for (int t = s_mid[i]; t < s_beg[i + 1]; ++t) di += (__popc(k & s_z[t]) & 1) ? -s_w[t] : s_w[t];
      } else {
        const int op = s_glob[i];
        const int sb = tb.poff[op], sm = tb.pmid[op], se = tb.poff[op + 1];
        for (int t = sb; t < sm; ++t) dr += (__popc(k & tb.pz[t]) & 1) ? -pw[t] : pw[t];
        for (int t = sm; t < se; ++t) di += (__popc(k & tb.pz[t]) & 1) ? -pw[t] : pw[t];
      }
      const C_t<R> p = psi[k ^ s_x[i]];
      // Re(conj(h) * D * p)
      const R ax = dr * p.x - di * p.y, ay = dr * p.y + di * p.x;
      const R val = h.x * ax + h.y * ay;
      if (sizeof(R) == 4) {
        R y = val - cmp[i], t = acc[i] + y;
        cmp[i] = (t - acc[i]) - y;
        acc[i] = t;
      } else {
        acc[i] += val;
      }
    }
  }
  double v[kOpsPerBlock];
#pragma unroll
  for (int i = 0; i < kOpsPerBlock; ++i) v[i] = (double)acc[i] - (double)cmp[i];
  // raw holds a whole number of chunks, so the tail chunk's unused slots are padding
  grid_sum<kOpsPerBlock>(v, partials + (size_t)blockIdx.y * gridDim.x * kOpsPerBlock,
                         counters + blockIdx.y, gridDim.x, blockIdx.x, raw + first, tot);
}

// Pool gradients for generators in LUT form.  blockIdx.y picks
// kOpsPerBlock operators in GOCP family order; blockIdx.x a range of
// kThreads * kPairsPerThread of each operator's enumerated touched pairs
// {b, b^x} (see PairEnum).  Operators are taken one after another (one
// accumulator per thread):
//   Re<H psi|A psi> over a pair = D(b) Re(conj(h_b) psi_{b^x}) + D(b^x) Re(conj(h_{b^x}) psi_b).
// Each block writes one FP64 partial per operator: part[pos * nbx + blockIdx.x].
// With `mask` set (nonzero octets of psi) a pair on which psi is zero at
// both ends adds nothing and is skipped before its loads.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_pool_grad_lut(DevTables tb, const C_t<R>* __restrict__ psi, const C_t<R>* __restrict__ hpsi,
                double* part, int nbx, const uint32_t* __restrict__ mask) {
  __shared__ LutDev<R> s_op[kOpsPerBlock];
  __shared__ PairEnum s_en[kOpsPerBlock];
  __shared__ double s_red[kWarps];
  const int first = blockIdx.y * kOpsPerBlock;
  const int nops = min(kOpsPerBlock, tb.M - first);
  const LutDev<R>* pl = (const LutDev<R>*)tb.plut;
  if (threadIdx.x < nops) {
    const int op = tb.porder[first + threadIdx.x];
    s_op[threadIdx.x] = pl[op];
    s_en[threadIdx.x] = tb.penum[op];
  }
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kThreads * kPairsPerThread;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 0; o < nops; ++o) {
    const LutDev<R>& L = s_op[o];
    const PairEnum& E = s_en[o];
    const uint64_t count = (uint64_t)E.ncodes << E.log2cnt;
    const uint32_t phx = L.fx & 7u, sgx = (L.fx >> 3) & 1u;
    R acc = 0, cmp = 0;
    if (base < count) {
#pragma unroll 4
      for (int jj = 0; jj < kPairsPerThread; ++jj) {
        const uint64_t q = base + (uint64_t)jj * kThreads + threadIdx.x;
        if (q >= count) break;
        uint32_t ph;
        const uint32_t b = enum_pair(E, (uint32_t)q, &ph);
        const uint32_t b2 = b ^ L.x;
        if (mask && !(octet_bit(mask, b) | octet_bit(mask, b2))) continue;
        const R l1 = L.lut[ph], l2 = L.lut[ph ^ phx];
        const uint32_t sg = __popc(b & L.z0) & 1u;
        const C_t<R> h1 = hpsi[b], h2 = hpsi[b2], p1 = psi[b], p2 = psi[b2];
        const R val = (sg ? -l1 : l1) * (h1.x * p2.x + h1.y * p2.y) +
                      ((sg ^ sgx) ? -l2 : l2) * (h2.x * p1.x + h2.y * p1.y);
        if (sizeof(R) == 4) {
          R y = val - cmp, t = acc + y;
          cmp = (t - acc) - y;
          acc = t;
        } else {
          acc += val;
        }
      }
    }
    double v = (double)acc - (double)cmp;
    v = warp_sum(v);
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += s_red[w];
      part[(size_t)(first + o) * nbx + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// ---- pool gradients driven by the live octets (full layout, LUT pool)
//
// The octets of psi that hold a nonzero amplitude (8.85 % at 24 qubits for
// the ADAPT states) are listed in index order (k_live_count, k_live_list);
// a thread takes one live octet, loads its 8 amplitudes of psi and H psi
// once, and for each generator of its block's chunk visits the octet's
// members k = 8o + i: as the base of a pair (bit s of k clear) always, as
// the partner only when the base octet is not live (then psi is zero there
// and the pair has no other visitor).  Pairs with psi zero at both ends are
// never visited; they add nothing.

constexpr int kLiveWordsPerThread = 8;

// counts[b] = live octets in the mask words of block b (2048 words each).
__global__ void __launch_bounds__(kThreads) k_live_count(const uint32_t* mask, uint32_t words, uint32_t* counts) {
  __shared__ uint32_t red[kWarps];
  const uint32_t w0 = (blockIdx.x * kThreads + threadIdx.x) * kLiveWordsPerThread;
  uint32_t c = 0;
  for (int q = 0; q < kLiveWordsPerThread; ++q)
    if (w0 + q < words) c += __popc(mask[w0 + q]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kWarps; ++w) t += red[w];
    counts[blockIdx.x] = t;
  }
}

// list[...] = the live octets in index order; list_len[0] = their number.
__global__ void __launch_bounds__(kThreads)
k_live_list(const uint32_t* mask, uint32_t words, const uint32_t* counts, uint32_t* list, uint32_t* list_len) {
  __shared__ uint32_t scan[kThreads];
  __shared__ uint32_t before;
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (uint32_t b = 0; b < blockIdx.x; ++b) t += counts[b];
    before = t;
    if (blockIdx.x == gridDim.x - 1) *list_len = t + counts[blockIdx.x];
  }
  const uint32_t w0 = (blockIdx.x * kThreads + threadIdx.x) * kLiveWordsPerThread;
  uint32_t c = 0;
  for (int q = 0; q < kLiveWordsPerThread; ++q)
    if (w0 + q < words) c += __popc(mask[w0 + q]);
  scan[threadIdx.x] = c;
  __syncthreads();
  for (int d = 1; d < kThreads; d <<= 1) {   // inclusive scan
    const uint32_t v = threadIdx.x >= d ? scan[threadIdx.x - d] : 0u;
    __syncthreads();
    scan[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t at = before + scan[threadIdx.x] - c;
  for (int q = 0; q < kLiveWordsPerThread; ++q) {
    if (w0 + q >= words) break;
    uint32_t m = mask[w0 + q];
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1u;
      list[at++] = (w0 + q) * 32u + (uint32_t)b;
    }
  }
}

int live_octets(const uint32_t* mask, int n, const LiveOctets& lv, cudaStream_t st) {
  if (n < 8 || !mask || !lv.list) return fail(GOCP_EINVAL, "live octets need n >= 8 and buffers");
  const uint32_t words = 1u << (n - 8);
  const int nb = (int)((words + kThreads * kLiveWordsPerThread - 1) / (kThreads * kLiveWordsPerThread));
  k_live_count<<<nb, kThreads, 0, st>>>(mask, words, lv.counts);
  k_live_list<<<nb, kThreads, 0, st>>>(mask, words, lv.counts, lv.list, lv.len);
  count_launches(2);
  return cuda_status(cudaGetLastError(), "k_live_list");
}

// ---- pool gradients driven by the nonzero amplitudes (full layout, LUT pool)
//
// raw_k = sum_b Re(conj((H psi)_b) D_k(b) psi_{b ^ x}) needs only the b with
// psi_{b ^ x} != 0, i.e. b = k' ^ x for the listed nonzero amplitudes psi(k')
// (amp_list); every such b is reached exactly once.  A block takes a slice
// of the list and its kOpsPerBlock generators one after the other (the
// slice stays in L1 across them); a thread and its warp sum in R, the
// block in FP64; (H psi)_b is read only where
// D_k(b) != 0.  Returns at once when the list is incomplete (more than acap
// amplitudes): the live-octet kernel then runs.
//
// complex128: the FP64 pipe is about 1/64 the width of FP32 here, and most
// (amplitude, generator) items have D_k(b) = 0.  The zero test and the sign
// work on the bits of D with integer instructions, and a warp packs its
// nonzero items (b, list index, signed D) into a shared-memory buffer and
// computes them 32 at a time with every lane busy, instead of running the
// FP64 products whenever any lane has a nonzero item.  A lane's items are
// summed in the same order either way except for that grouping, so the
// gradients differ only by the rounding of the per-thread sums.
struct __align__(16) GradItem {
  uint32_t b, l;
  double d;
};
constexpr int kGradCap = 64;   // items a warp's buffer holds: < 32 left after a flush + 32 new

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_pool_grad_amp(DevTables tb, const C_t<R>* __restrict__ hpsi, const uint32_t* __restrict__ aidx,
                const C_t<R>* __restrict__ aval, const uint32_t* __restrict__ alen, uint32_t acap, double* part,
                int nbx) {
  if (*alen > acap) return;
  __shared__ LutDev<R> s_op[kOpsPerBlock];
  __shared__ double s_red[kOpsPerBlock][kWarps];
  if constexpr (sizeof(R) == 8) {
    __shared__ GradItem s_items[kWarps][kGradCap];
    const int first = blockIdx.y * kOpsPerBlock;
    const int nops = min(kOpsPerBlock, tb.M - first);
    if (threadIdx.x < nops) s_op[threadIdx.x] = ((const LutDev<R>*)tb.plut)[tb.porder[first + threadIdx.x]];
    __syncthreads();
    const uint32_t n = *alen;
    const uint32_t per = (n + nbx - 1) / nbx;
    const uint32_t l0 = blockIdx.x * per, l1 = min(n, l0 + per);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    GradItem* wb = s_items[warp];
    auto flush = [&](uint32_t at, bool on, double& acc) {
      __syncwarp();
      if (on) {
        const GradItem e = wb[at];
        const C_t<R> p = aval[e.l], h = hpsi[e.b];
        acc += e.d * ((double)h.x * p.x + (double)h.y * p.y);
      }
      __syncwarp();
    };
    for (int o = 0; o < nops; ++o) {
      const LutDev<R>& L = s_op[o];
      double acc = 0.0;
      uint32_t cnt = 0;   // items in wb (warp-uniform)
      // the warp walks the slice together so that the ballots see every lane
      for (uint32_t l = l0 + (uint32_t)threadIdx.x - (uint32_t)lane; l < l1; l += kThreads) {
        const uint32_t li = l + (uint32_t)lane;
        const bool in = li < l1;
        const uint32_t b = (in ? aidx[li] : 0u) ^ L.x;
        const long long db = __double_as_longlong((double)L.lut[lut_phi(L, b)]);
        const bool nz = in && (db << 1) != 0ll;
        const uint32_t m = __ballot_sync(0xffffffffu, nz);
        if (nz) {
          GradItem e;
          e.b = b;
          e.l = li;
          e.d = __longlong_as_double(db ^ ((long long)(__popc(b & L.z0) & 1) << 63));
          wb[cnt + (uint32_t)__popc(m & lt)] = e;
        }
        cnt += (uint32_t)__popc(m);
        if (cnt >= 32u) {
          cnt -= 32u;
          flush(cnt + (uint32_t)lane, true, acc);
        }
      }
      if (cnt) flush((uint32_t)lane, (uint32_t)lane < cnt, acc);
      acc = warp_sum(acc);
      if (lane == 0) s_red[o][warp] = acc;
    }
    __syncthreads();
    if (threadIdx.x < nops) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += s_red[threadIdx.x][w];
      part[(size_t)(first + threadIdx.x) * nbx + blockIdx.x] = t;
    }
    return;
  }
  const int first = blockIdx.y * kOpsPerBlock;
  const int nops = min(kOpsPerBlock, tb.M - first);
  if (threadIdx.x < nops) s_op[threadIdx.x] = ((const LutDev<R>*)tb.plut)[tb.porder[first + threadIdx.x]];
  __syncthreads();
  const uint32_t n = *alen;
  const uint32_t per = (n + nbx - 1) / nbx;
  const uint32_t l0 = blockIdx.x * per, l1 = min(n, l0 + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 0; o < nops; ++o) {
    const LutDev<R>& L = s_op[o];
    R acc = R(0);
    for (uint32_t l = l0 + threadIdx.x; l < l1; l += kThreads) {
      const uint32_t b = aidx[l] ^ L.x;
      const R d = L.lut[lut_phi(L, b)];
      if (d == R(0)) continue;
      const C_t<R> p = aval[l], h = hpsi[b];
      acc += ((__popc(b & L.z0) & 1) ? -d : d) * (h.x * p.x + h.y * p.y);
    }
    // the warp's sum in R (FP64 is a slow pipe here), the block's in FP64
    for (int q = 16; q > 0; q >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, q);
    if (lane == 0) s_red[o][warp] = (double)acc;
  }
  __syncthreads();
  if (threadIdx.x < nops) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += s_red[threadIdx.x][w];
    part[(size_t)(first + threadIdx.x) * nbx + blockIdx.x] = t;
  }
}

// gate set: returns at once when *gate <= gate_max (k_pool_grad_amp runs).
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_pool_grad_live(DevTables tb, const C_t<R>* __restrict__ psi, const C_t<R>* __restrict__ hpsi,
                 const uint32_t* __restrict__ mask, const uint32_t* __restrict__ list,
                 const uint32_t* __restrict__ list_len, double* part, int nbx, const uint32_t* gate,
                 uint32_t gate_max) {
  if (gate && *gate <= gate_max) return;
  __shared__ LutDev<R> s_op[kOpsPerBlock];
  __shared__ double s_red[kWarps];
  const int first = blockIdx.y * kOpsPerBlock;
  const int nops = min(kOpsPerBlock, tb.M - first);
  if (threadIdx.x < nops) s_op[threadIdx.x] = ((const LutDev<R>*)tb.plut)[tb.porder[first + threadIdx.x]];
  __syncthreads();
  const uint32_t n_live = *list_len;
  const uint32_t per = (n_live + nbx - 1) / nbx;
  const uint32_t l0 = blockIdx.x * per, l1 = min(n_live, l0 + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 0; o < nops; ++o) {
    const LutDev<R>& L = s_op[o];
    const uint32_t phx = L.fx & 7u, sgx = (L.fx >> 3) & 1u;
    R acc = 0, cmp = 0;
    for (uint32_t l = l0 + threadIdx.x; l < l1; l += kThreads) {
      const uint32_t k0 = list[l] * kAmpsH;
      R a = 0;
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) {
        const uint32_t k = k0 + i;
        const uint32_t ph = lut_phi(L, k), sg = __popc(k & L.z0) & 1u;
        if (!((k >> L.s) & 1u)) {
          // k is the base of pair (k, k ^ x)
          const R l1 = L.lut[ph], l2 = L.lut[ph ^ phx];
          if (l1 == R(0) && l2 == R(0)) continue;
          const uint32_t kp = k ^ L.x;
          const C_t<R> pk = psi[k], hk = hpsi[k], pp = psi[kp], hp = hpsi[kp];
          a += (sg ? -l1 : l1) * (hk.x * pp.x + hk.y * pp.y) + ((sg ^ sgx) ? -l2 : l2) * (hp.x * pk.x + hp.y * pk.y);
        } else {
          // k is the partner of base b = k ^ x: visited here only when b's octet is not live (psi_b = 0)
          const uint32_t b = k ^ L.x;
          if (octet_bit(mask, b)) continue;
          const uint32_t phb = ph ^ phx, sgb = sg ^ sgx;
          const R l1 = L.lut[phb];
          if (l1 == R(0)) continue;
          const C_t<R> pk = psi[k], hb = hpsi[b];
          a += (sgb ? -l1 : l1) * (hb.x * pk.x + hb.y * pk.y);
        }
      }
      if (sizeof(R) == 4) {
        const R y = a - cmp, t = acc + y;
        cmp = (t - acc) - y;
        acc = t;
      } else {
        acc += a;
      }
    }
    const double v = warp_sum((double)acc - (double)cmp);
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += s_red[w];
      part[(size_t)(first + o) * nbx + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// raw[i] = sum over the nbx block partials of operator i (family order), in
// a fixed order: one warp per operator.
__global__ void k_pool_reduce(const double* part, int nbx, int m, double* raw) {
  const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  double s = 0.0;
  for (int b = lane; b < nbx; b += 32) s += part[(size_t)i * nbx + b];
  s = warp_sum(s);
  if (lane == 0) raw[i] = s;
}

// ------------------------------------------------------------ batched stages

// One work item of a batched launch (device copy of a StageItem).
struct BatchItemDev {
  DevTables t;
  const int32_t* ops;
  const double* theta;
  double* coefs;
  void* psi;
  void* lam;
  double* partials;
  unsigned int* counter;
  double* scal;
  double* dtheta;
  int32_t* err;
  double identity;
  uint32_t ref_index;
  int n_ops;
  int j;
  int nb;
};

struct BatchIndex {
  int n;
  int start[kMaxBatchItems + 1];   // first block of each item
};

__device__ __forceinline__ int find_item(const BatchIndex& ix, int& bid) {
  int lo = 0, hi = ix.n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (ix.start[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  bid = blockIdx.x - ix.start[lo];
  return lo;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_stage_setup(const BatchItemDev* items, BatchIndex ix) {
  int bid;
  const BatchItemDev& it = items[find_item(ix, bid)];
  setup_body<R>((C_t<R>*)it.psi, it.t.n, it.ref_index, it.theta, it.n_ops, it.coefs, bid, it.nb);
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_stage_forward(const BatchItemDev* items, BatchIndex ix) {
  int bid;
  const BatchItemDev& it = items[find_item(ix, bid)];
  taylor_body<R>(it.t, it.ops, it.coefs, it.j, (C_t<R>*)it.psi, it.err, bid, it.nb);
}

template <typename R>
__global__ void __launch_bounds__(kThreads, 2) k_stage_energy(const BatchItemDev* items, BatchIndex ix) {
  int bid;
  const BatchItemDev& it = items[find_item(ix, bid)];
  apply_body<R>(it.t, (const C_t<R>*)it.psi, (C_t<R>*)it.lam, it.identity, it.partials, it.counter,
                it.scal, bid, it.nb);
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_stage_residual(const BatchItemDev* items, BatchIndex ix) {
  int bid;
  const BatchItemDev& it = items[find_item(ix, bid)];
  residual_body<R>((const C_t<R>*)it.psi, (C_t<R>*)it.lam, it.t.n, it.scal, bid, it.nb);
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_stage_backward(const BatchItemDev* items, BatchIndex ix) {
  int bid;
  const BatchItemDev& it = items[find_item(ix, bid)];
  adjoint_body<R>(it.t, it.ops, it.coefs, it.j, (C_t<R>*)it.psi, (C_t<R>*)it.lam, it.partials,
                  it.counter, it.dtheta, it.err, bid, it.nb);
}

// The whole forward chain / backward sweep of one small item per block
// (on-chip chains; the items' states fit kSmemStateBytes, two states for the
// backward sweep).
template <typename R>
__global__ void __launch_bounds__(kSmemThreads, 1) k_stage_forward_all(const BatchItemDev* items) {
  extern __shared__ __align__(16) uint8_t cs_raw[];
  const BatchItemDev& it = items[blockIdx.x];
  taylor_chain_smem_body<R>(it.t, it.ops, it.coefs, it.n_ops, (C_t<R>*)it.psi, it.err, nullptr,
                            reinterpret_cast<C_t<R>*>(cs_raw));
}

template <typename R>
__global__ void __launch_bounds__(kSmemThreads, 1) k_stage_backward_all(const BatchItemDev* items) {
  extern __shared__ __align__(16) uint8_t cs_raw[];
  const BatchItemDev& it = items[blockIdx.x];
  adjoint_chain_smem_body<R>(it.t, it.ops, it.coefs, it.n_ops, (C_t<R>*)it.psi, (C_t<R>*)it.lam, it.dtheta,
                             it.err, reinterpret_cast<C_t<R>*>(cs_raw));
}

// ------------------------------------------------------------ upload

namespace {

template <typename T>
int dalloc(DeviceTables& d, T** p, size_t count, size_t& bytes) {
  if (count == 0) count = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) return cuda_status(e, "cudaMalloc");
  d.allocs.push_back(q);
  bytes += count * sizeof(T);
  *p = (T*)q;
  return GOCP_OK;
}

template <typename T>
int upload(DeviceTables& d, T** p, const std::vector<T>& h, size_t& bytes) {
  int rc = dalloc(d, p, h.size(), bytes);
  if (rc) return rc;
  if (h.empty()) return GOCP_OK;
  return cuda_status(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice),
                     "cudaMemcpy");
}

inline int parity32(uint32_t v) { return __builtin_popcount(v) & 1; }

// Effective weight of c i^phase X^x Z^z at output index k:
//   c i^phase (-1)^popc(x & z) -- real if phase is even, imaginary if odd.
inline double eff_weight(double c, int phase, uint32_t x, uint32_t z, bool* imag) {
  double w = (phase & 2) ? -c : c;
  if (parity32(x & z)) w = -w;
  *imag = phase & 1;
  return w;
}

// LUT descriptor of one x-group with real weights w (effective weights at
// the output index, as in the term tables); false when the rank exceeds 3.
template <typename R>
bool make_lut(uint32_t x, const std::vector<uint32_t>& z, const std::vector<double>& w, LutDev<R>* out) {
  if (z.empty() || x == 0) return false;
  LutForm f = lut_form(z.data(), w.data(), (int)z.size());
  if (!f.ok) return false;
  LutDev<R> L;
  std::memset(&L, 0, sizeof(L));
  L.x = x;
  L.z0 = f.z0;
  L.v0 = f.d > 0 ? f.v[0] : 0u;
  L.v1 = f.d > 1 ? f.v[1] : 0u;
  L.v2 = f.d > 2 ? f.v[2] : 0u;
  const uint32_t phx = (uint32_t)parity32(x & L.v0) | ((uint32_t)parity32(x & L.v1) << 1) |
                       ((uint32_t)parity32(x & L.v2) << 2);
  L.fx = phx | ((uint32_t)parity32(x & f.z0) << 3);
  L.s = __builtin_ctz(x);
  for (int i = 0; i < 8; ++i) L.lut[i] = (R)(i < (1 << f.d) ? f.lut[i] : 0.0);
  *out = L;
  return true;
}

// Touched-pair enumeration of a LUT-form generator (see PairEnum).
bool make_enum(const LutForm& f, uint32_t x, int n, PairEnum* out) {
  const int s = __builtin_ctz(x);
  const uint32_t sbit = 1u << s;
  uint32_t R[3], Cm[3], dep[3];
  int piv[3], r = 0, ndep = 0;
  for (int i = 0; i < f.d; ++i) {
    uint32_t v = f.v[i] & ~sbit, c = 1u << i;
    for (int k = 0; k < r; ++k)
      if ((v >> piv[k]) & 1u) { v ^= R[k]; c ^= Cm[k]; }
    if (v == 0) { dep[ndep++] = c; continue; }   // rows in c sum to zero on b with bit s clear
    const int p = 31 - __builtin_clz(v);
    for (int k = 0; k < r; ++k)
      if ((R[k] >> p) & 1u) { R[k] ^= v; Cm[k] ^= c; }
    R[r] = v; Cm[r] = c; piv[r] = p; ++r;
  }
  const uint32_t phx = (uint32_t)parity32(x & f.v[0]) | ((uint32_t)parity32(x & f.v[1]) << 1) |
                       ((uint32_t)parity32(x & f.v[2]) << 2);
  PairEnum e;
  std::memset(&e, 0, sizeof(e));
  int nc = 0;
  uint64_t codes = 0;
  for (uint32_t c = 0; c < (1u << f.d); ++c) {
    bool ok = true;
    for (int q = 0; q < ndep; ++q) ok = ok && !parity32(c & dep[q]);
    if (!ok) continue;
    const double l1 = f.lut[c], l2 = f.lut[(c ^ phx) & ((1u << f.d) - 1)];
    if (l1 == 0.0 && l2 == 0.0) continue;
    uint32_t red = 0;
    for (int k = 0; k < r; ++k) red |= (uint32_t)parity32(c & Cm[k]) << k;
    codes |= (uint64_t)(red | (c << 3)) << (8 * nc);
    ++nc;
  }
  if (nc == 0) return false;
  std::vector<int> ex{s};
  for (int k = 0; k < r; ++k) ex.push_back(piv[k]);
  std::sort(ex.begin(), ex.end());
  for (size_t q = 0; q < ex.size(); ++q) e.excl |= (uint32_t)ex[q] << (8 * q);
  for (int k = 0; k < r; ++k) {
    e.piv |= (uint32_t)piv[k] << (8 * k);
    e.pmask[k] = R[k] & ~(1u << piv[k]);
  }
  e.codes = (uint32_t)codes;
  e.codes_hi = (uint32_t)(codes >> 32);
  e.nex = (uint8_t)ex.size();
  e.r = (uint8_t)r;
  e.ncodes = (uint8_t)nc;
  e.log2cnt = (uint8_t)(n - 1 - r);
  *out = e;
  return true;
}

// LUT descriptor of one H x-group for the octet layout of the H psi kernel.
template <typename R>
bool make_hlut(uint32_t x, const std::vector<uint32_t>& z, const std::vector<double>& w, HLut<R>* out) {
  if (z.empty() || x == 0) return false;
  LutForm f = lut_form(z.data(), w.data(), (int)z.size());
  if (!f.ok) return false;
  HLut<R> L;
  std::memset(&L, 0, sizeof(L));
  L.x = x;
  L.z0 = f.z0;
  L.v0 = f.d > 0 ? f.v[0] : 0u;
  L.v1 = f.d > 1 ? f.v[1] : 0u;
  L.v2 = f.d > 2 ? f.v[2] : 0u;
  uint32_t reg = 0;
  for (uint32_t i = 0; i < 8; ++i) {
    const uint32_t code = (uint32_t)parity32(i & L.v0) | ((uint32_t)parity32(i & L.v1) << 1) |
                          ((uint32_t)parity32(i & L.v2) << 2) | ((uint32_t)parity32(i & f.z0) << 3);
    reg |= code << (4 * i);
  }
  L.reg = reg;
  for (int c = 0; c < 16; ++c) {
    const int ph = c & 7;
    const double val = ph < (1 << f.d) ? f.lut[ph] : 0.0;
    L.lut16[c] = (R)((c & 8) ? -val : val);
  }
  *out = L;
  return true;
}

// The exact pair structure of a term-list group with real weights (see
// TiledGroup): a vector delta != 0 and a sign such that every term (z, w) has
// the partner (z ^ delta, sign * w), found among delta = z_0 ^ z_t.  Returns
// delta = 0 when there is none (or the group has imaginary terms); else the
// terms with bit lowbit(delta) of z clear, sorted into Walsh buckets by
// z & 7, and their bucket sizes.
template <typename R>
struct PairedTerms {
  uint32_t delta = 0, neg = 0;
  uint64_t bk = ~0ull;
  std::vector<uint32_t> z;
  std::vector<R> w;
};

template <typename R>
PairedTerms<R> paired_terms(const std::vector<uint32_t>& tz, const std::vector<R>& tw, int32_t beg,
                             int32_t mid, int32_t end) {
  PairedTerms<R> out;
  const int cnt = end - beg;
  if (mid != end || cnt < 2 || (cnt & 1)) return out;
  std::vector<std::pair<uint32_t, R>> terms;
  for (int32_t t = beg; t < end; ++t) terms.push_back({tz[t], tw[t]});
  std::sort(terms.begin(), terms.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  auto find = [&](uint32_t z, R* w) {
    auto it = std::lower_bound(terms.begin(), terms.end(), z,
                               [](const std::pair<uint32_t, R>& a, uint32_t v) { return a.first < v; });
    if (it == terms.end() || it->first != z) return false;
    *w = it->second;
    return true;
  };
  for (int c = 1; c < cnt && !out.delta; ++c) {
    const uint32_t d = terms[0].first ^ terms[c].first;
    for (int sgn = 0; sgn < 2 && !out.delta; ++sgn) {
      bool ok = true;
      for (const auto& tm : terms) {
        R w2;
        if (!find(tm.first ^ d, &w2) || w2 != (sgn ? -tm.second : tm.second)) {
          ok = false;
          break;
        }
      }
      if (ok) {
        out.delta = d;
        out.neg = (uint32_t)sgn;
      }
    }
  }
  if (!out.delta) return out;
  const uint32_t low = out.delta & (~out.delta + 1u);
  int nb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int m = 0; m < 8; ++m)
    for (const auto& tm : terms)
      if (!(tm.first & low) && (tm.first & 7u) == (uint32_t)m) {
        out.z.push_back(tm.first);
        out.w.push_back(tm.second);
        ++nb[m];
      }
  out.bk = 0;
  for (int m = 0; m < 8; ++m) {
    if (nb[m] > 255) {
      out.delta = 0;   // a bucket too large for the packed sizes: keep the group unpaired
      out.bk = ~0ull;
      out.z.clear();
      out.w.clear();
      return out;
    }
    out.bk |= (uint64_t)nb[m] << (8 * m);
  }
  return out;
}

// Cuts the off-diagonal groups into the pieces of the tiled H psi kernel
// (see TiledHead).  hl and the term-list groups come sorted by (x & 7, x),
// an order each piece keeps.  Leaves t.n_pieces = 0 (the untiled kernel
// serves the problem) when n is below the tile size or a single group does
// not fit one blob.
template <typename R>
int build_tiled(int n, const std::vector<HLut<R>>& hl, const std::vector<uint32_t>& gx,
                const std::vector<int32_t>& goff, const std::vector<int32_t>& gmid,
                const std::vector<uint64_t>& gbk, const std::vector<uint32_t>& tz,
                const std::vector<R>& tw, DeviceTables& d, size_t& bytes) {
  constexpr int LB = TiledBits<R>::LB;
  constexpr uint32_t octets = 1u << (LB - 3);
  static_assert(kTiledBlobBytes / sizeof(TiledGroup) < 4096, "run bounds of a piece fit 12 bits");
  d.t.n_pieces = 0;
  if (n < LB) return GOCP_OK;
  auto a16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
  auto blob_size = [&](size_t nl, size_t ng, size_t nt) {
    return sizeof(TiledHead) + nl * sizeof(HLut<R>) + ng * sizeof(TiledGroup) + a16(nt * 4) +
           a16(nt * sizeof(R));
  };
  // segments by x >> LB: x_hi != 0 ascending, then x_hi = 0
  std::vector<uint32_t> his;
  for (const HLut<R>& L : hl) his.push_back(L.x >> LB);
  for (uint32_t x : gx) his.push_back(x >> LB);
  his.push_back(0u);
  std::sort(his.begin(), his.end());
  his.erase(std::unique(his.begin(), his.end()), his.end());
  std::rotate(his.begin(), his.begin() + 1, his.end());   // 0 (the smallest) last
  // terms each group keeps in the blob (half of them when paired)
  std::vector<size_t> stored(gx.size());
  for (size_t g = 0; g < gx.size(); ++g) {
    const auto pr = paired_terms<R>(tz, tw, goff[g], gmid[g], goff[g + 1]);
    stored[g] = pr.delta ? pr.z.size() : (size_t)(goff[g + 1] - goff[g]);
  }
  std::vector<uint8_t> blob;
  std::vector<TiledPiece> pieces;
  for (uint32_t hi : his) {
    std::vector<int> ls, ts;
    for (int g = 0; g < (int)hl.size(); ++g)
      if ((hl[g].x >> LB) == hi) ls.push_back(g);
    for (int g = 0; g < (int)gx.size(); ++g)
      if ((gx[g] >> LB) == hi) ts.push_back(g);
    // LUT groups by kernel variant (flip class, x & 7), then x
    auto lut_key = [&](int g) { return (int)(tiled_flip_class(hl[g].reg) * 8u + (hl[g].x & 7u)); };
    std::stable_sort(ls.begin(), ls.end(), [&](int a, int b) { return lut_key(a) < lut_key(b); });
    size_t li = 0, ti = 0;
    do {
      std::vector<int> pl, pt;
      size_t nt = 0;
      int lruns = 0, truns = 0;
      while (li < ls.size() && blob_size(pl.size() + 1, 0, 0) <= kTiledBlobBytes) {
        const bool fresh = pl.empty() || lut_key(ls[li]) != lut_key(pl.back());
        if (fresh && lruns == kTiledRuns - 8) break;   // keep 8 runs for the term lists
        lruns += fresh;
        pl.push_back(ls[li++]);
      }
      while (ti < ts.size()) {
        const int g = ts[ti];
        const size_t add = stored[g];
        if (blob_size(pl.size(), pt.size() + 1, nt + add) > kTiledBlobBytes) break;
        const bool fresh = pt.empty() || (gx[g] & 7u) != (gx[pt.back()] & 7u);
        if (fresh && lruns + truns == kTiledRuns) break;
        truns += fresh;
        pt.push_back(g);
        nt += add;
        ++ti;
      }
      if (pl.empty() && pt.empty() && (li < ls.size() || ti < ts.size())) return GOCP_OK;
      TiledHead h;
      std::memset(&h, 0, sizeof(h));
      h.n_lut = (uint32_t)pl.size();
      const size_t z_off = sizeof(TiledHead) + pl.size() * sizeof(HLut<R>) + pt.size() * sizeof(TiledGroup);
      h.z_off = (uint32_t)z_off;
      h.w_off = (uint32_t)(z_off + a16(nt * 4));
      for (int kind = 0; kind < 2; ++kind) {
        const int cnt = kind == 0 ? (int)pl.size() : (int)pt.size();
        auto sel_of = [&](int q) { return kind == 0 ? lut_key(pl[q]) : 64 + (int)(gx[pt[q]] & 7u); };
        for (int q = 0; q < cnt;) {
          int e = q;
          while (e < cnt && sel_of(e) == sel_of(q)) ++e;
          h.run[h.n_runs++] = (uint32_t)q | ((uint32_t)e << 12) | ((uint32_t)sel_of(q) << 24);
          q = e;
        }
      }
      const size_t total = blob_size(pl.size(), pt.size(), nt);
      const size_t off = blob.size();
      blob.resize(off + total, 0);
      uint8_t* b = blob.data() + off;
      std::memcpy(b, &h, sizeof(h));
      size_t w = sizeof(TiledHead);
      for (int g : pl) {
        HLut<R> L = hl[g];
        L.pad0 = tiled_swz<R>((L.x >> 3) & (octets - 1));
        L.pad1 = (L.x >> 3) & (octets - 1);
        std::memcpy(b + w, &L, sizeof(HLut<R>));
        w += sizeof(HLut<R>);
      }
      uint32_t tcur = 0;
      std::vector<uint32_t> zz;
      std::vector<R> ww;
      for (int g : pt) {
        TiledGroup tg;
        std::memset(&tg, 0, sizeof(tg));
        tg.x = gx[g];
        tg.xa = tiled_swz<R>((gx[g] >> 3) & (octets - 1));
        tg.pad = (gx[g] >> 3) & (octets - 1);
        const auto pr = paired_terms<R>(tz, tw, goff[g], gmid[g], goff[g + 1]);
        tg.tb = tcur;
        if (pr.delta) {
          tg.delta = pr.delta;
          tg.neg = pr.neg;
          tg.bk = pr.bk;
          tg.tm = tg.te = tcur + (uint32_t)pr.z.size();
          zz.insert(zz.end(), pr.z.begin(), pr.z.end());
          ww.insert(ww.end(), pr.w.begin(), pr.w.end());
        } else {
          tg.tm = tcur + (uint32_t)(gmid[g] - goff[g]);
          tg.te = tcur + (uint32_t)(goff[g + 1] - goff[g]);
          tg.bk = gbk[g];
          for (int32_t t = goff[g]; t < goff[g + 1]; ++t) {
            zz.push_back(tz[t]);
            ww.push_back(tw[t]);
          }
        }
        tcur = tg.te;
        std::memcpy(b + w, &tg, sizeof(tg));
        w += sizeof(tg);
      }
      if (!zz.empty()) {
        std::memcpy(b + h.z_off, zz.data(), zz.size() * 4);
        std::memcpy(b + h.w_off, ww.data(), ww.size() * sizeof(R));
      }
      TiledPiece pc;
      pc.xhi = hi;
      pc.off = (uint32_t)off;
      pc.bytes = (uint32_t)total;
      pc.pad = 0;
      pieces.push_back(pc);
    } while (li < ls.size() || ti < ts.size());
  }
  // the scatter kernel numbers a tile's work units piece by piece in this
  // order (costliest first), so that the units left at the end of a tile are
  // short ones
  std::vector<uint32_t> porder(pieces.size());
  for (size_t i = 0; i < porder.size(); ++i) porder[i] = (uint32_t)i;
  std::stable_sort(porder.begin(), porder.end(),
                   [&](uint32_t a, uint32_t b) { return pieces[a].bytes > pieces[b].bytes; });
  // complex128: the LUT entries and term weights again, as fixed-point
  // integers round(w 2^Fd) at their own offsets (the scatter kernel forms
  // its products in integers, see q_mul there).  Fd = 62 - e with
  // dmax < 2^e, so that every |w| 2^Fd, and every group's sum of |w| 2^Fd,
  // stays below 2^62.
  std::vector<uint8_t> wfix;
  int fd = 0;
  if constexpr (sizeof(R) == 8) {
    if (d.t.dmax > 0.0) {
      int e;
      std::frexp(d.t.dmax, &e);   // dmax < 2^e
      fd = 62 - e;
    }
    auto put = [&](size_t at) {
      double v;
      std::memcpy(&v, blob.data() + at, sizeof(v));
      const long long q = std::llround(std::ldexp(v, fd));
      std::memcpy(wfix.data() + at, &q, sizeof(q));
    };
    wfix.assign(blob.size(), 0);
    for (const TiledPiece& pc : pieces) {
      TiledHead h;
      std::memcpy(&h, blob.data() + pc.off, sizeof(h));
      for (uint32_t g = 0; g < h.n_lut; ++g)
        for (int c = 0; c < 16; ++c)
          put(pc.off + sizeof(TiledHead) + g * sizeof(HLut<R>) + offsetof(HLut<R>, lut16) + c * sizeof(R));
      for (uint32_t o = h.w_off; o + sizeof(R) <= pc.bytes; o += sizeof(R)) put(pc.off + o);
    }
  }
  uint8_t* dblob;
  TiledPiece* dpiece;
  uint32_t* dporder;
  int rc;
  if (!wfix.empty()) {
    uint8_t* dw;
    if ((rc = upload(d, &dw, wfix, bytes))) return rc;
    d.t.twfix = dw;
    d.t.twscale = std::ldexp(1.0, 63 - fd);
  }
  if ((rc = upload(d, &dblob, blob, bytes)) || (rc = upload(d, &dpiece, pieces, bytes)) ||
      (rc = upload(d, &dporder, porder, bytes)) ||
      (rc = dalloc(d, &d.t.tflags, ((size_t)1 << (n - LB)) / 32 + 1, bytes)) ||
      (rc = dalloc(d, &d.live.toff, ((size_t)1 << (n - LB)) + 1, bytes)) ||
      (rc = dalloc(d, &d.live.aidx, (size_t)1 << (n - 2), bytes)) ||
      (rc = dalloc(d, reinterpret_cast<C_t<R>**>(&d.live.aval), (size_t)1 << (n - 2), bytes)) ||
      (rc = dalloc(d, &d.live.alen, 1, bytes)) || (rc = dalloc(d, &d.live.acounts, ((((size_t)1 << (n - 5)) + 255) / 256) + 1, bytes)) ||
      (rc = dalloc(d, &d.live.amax, 1, bytes)))
    return rc;
  d.live.acap = 1u << (n - 2);
  // few output tiles (below 512: up to 21 qubits complex64, 20 complex128):
  // global accumulators for the scatter kernel's blocks that share a tile,
  // zero between calls
  const size_t ntiles = (size_t)1 << (n - LB);
  if (ntiles < 512) {
    const size_t words = ntiles * (size_t)octets * 16u;
    if ((rc = dalloc(d, &d.live.gacc, words, bytes)) || (rc = dalloc(d, &d.live.tdone, ntiles, bytes))) return rc;
    if ((rc = cuda_status(cudaMemset(d.live.gacc, 0, words * sizeof(unsigned long long)), "zero gacc")) ||
        (rc = cuda_status(cudaMemset(d.live.tdone, 0, ntiles * sizeof(unsigned int)), "zero tdone")))
      return rc;
    d.live.gtiles = (uint32_t)ntiles;
  }
  d.t.tblob = dblob;
  d.t.tpiece = dpiece;
  d.t.tporder = dporder;
  d.t.n_pieces = (int)pieces.size();
  return GOCP_OK;
}

template <typename R>
int upload_typed(Problem& p, DeviceTables& d, size_t& bytes, double* identity) {
  const PauliTerms& H = p.H;
  // ---- Hamiltonian: identity apart, diagonal group apart, off-diagonal
  // groups in LUT form or as term lists, each sorted by (x & 7, x)
  struct TermGroup {
    uint32_t x;
    std::vector<uint32_t> zr, zi;
    std::vector<R> wr, wi;
  };
  std::vector<uint32_t> dz_r, dz_i;
  std::vector<R> dw_r, dw_i;
  std::vector<HLut<R>> hl;
  std::vector<TermGroup> tgs;
  double ident = 0.0;
  size_t i = 0;
  while (i < H.size()) {
    size_t j = i;
    while (j < H.size() && H.x[j] == H.x[i]) ++j;
    TermGroup tg;
    tg.x = H.x[i];
    std::vector<double> wr64;
    for (size_t t = i; t < j; ++t) {
      bool imag = false;
      double w = eff_weight(H.coeff[t], H.phase[t], H.x[t], H.z[t], &imag);
      if (H.x[t] == 0 && H.z[t] == 0 && !imag) {
        ident += w;
        continue;
      }
      (imag ? tg.zi : tg.zr).push_back(H.z[t]);
      (imag ? tg.wi : tg.wr).push_back((R)w);
      if (!imag) wr64.push_back(w);
    }
    HLut<R> L;
    if (H.x[i] == 0) {
      dz_r = tg.zr;
      dw_r = tg.wr;
      dz_i = tg.zi;
      dw_i = tg.wi;
    } else if (tg.zi.empty() && make_hlut<R>(H.x[i], tg.zr, wr64, &L)) {
      hl.push_back(L);
    } else if (!tg.zr.empty() || !tg.zi.empty()) {
      tgs.push_back(std::move(tg));
    }
    i = j;
  }
  *identity = ident;
  std::stable_sort(hl.begin(), hl.end(), [](const HLut<R>& a, const HLut<R>& b) {
    return (a.x & 7u) != (b.x & 7u) ? (a.x & 7u) < (b.x & 7u) : a.x < b.x;
  });
  std::stable_sort(tgs.begin(), tgs.end(), [](const TermGroup& a, const TermGroup& b) {
    return (a.x & 7u) != (b.x & 7u) ? (a.x & 7u) < (b.x & 7u) : a.x < b.x;
  });
  // LUT chunks: runs of equal x & 7 cut every kLutChunkH groups
  std::vector<int32_t> lchunk{0};
  std::vector<uint8_t> lchunk_xl;
  for (int g = 0; g < (int)hl.size();) {
    int h = g;
    while (h < (int)hl.size() && h - g < kLutChunkH && (hl[h].x & 7u) == (hl[g].x & 7u)) ++h;
    lchunk.push_back(h);
    lchunk_xl.push_back((uint8_t)(hl[g].x & 7u));
    g = h;
  }
  // term-list groups flattened; chunks fit the shared-memory stage and never
  // mix two values of x & 7 (a single oversized group is its own chunk)
  std::vector<uint32_t> gx, tz;
  std::vector<int32_t> goff, gmid;
  std::vector<R> tw;
  std::vector<uint64_t> gbk;
  for (TermGroup& tg : tgs) {
    uint64_t bk = ~0ull;
    if (tg.zi.empty()) {
      std::vector<size_t> idx(tg.zr.size());
      for (size_t q = 0; q < idx.size(); ++q) idx[q] = q;
      std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return (tg.zr[a] & 7u) < (tg.zr[b] & 7u); });
      std::vector<uint32_t> zs2;
      std::vector<R> ws2;
      int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (size_t q : idx) {
        zs2.push_back(tg.zr[q]);
        ws2.push_back(tg.wr[q]);
        ++cnt[tg.zr[q] & 7u];
      }
      bool fits = true;
      for (int m = 0; m < 8; ++m) fits = fits && cnt[m] <= 255;
      if (fits) {
        tg.zr.swap(zs2);
        tg.wr.swap(ws2);
        bk = 0;
        for (int m = 0; m < 8; ++m) bk |= (uint64_t)cnt[m] << (8 * m);
      }
    }
    gbk.push_back(bk);
    gx.push_back(tg.x);
    goff.push_back((int32_t)tz.size());
    tz.insert(tz.end(), tg.zr.begin(), tg.zr.end());
    tw.insert(tw.end(), tg.wr.begin(), tg.wr.end());
    gmid.push_back((int32_t)tz.size());
    tz.insert(tz.end(), tg.zi.begin(), tg.zi.end());
    tw.insert(tw.end(), tg.wi.begin(), tg.wi.end());
  }
  goff.push_back((int32_t)tz.size());
  const int G = (int)gx.size();
  std::vector<int32_t> chunk{0};
  std::vector<uint8_t> chunk_xl;
  for (int g = 0; g < G;) {
    int h = g;
    while (h < G && h - g < kChunkGroups && goff[h + 1] - goff[g] <= kChunkTerms &&
           (gx[h] & 7u) == (gx[g] & 7u))
      ++h;
    if (h == g) h = g + 1;
    chunk.push_back(h);
    chunk_xl.push_back((uint8_t)(gx[g] & 7u));
    g = h;
  }
  std::vector<uint32_t> dz(dz_r);
  dz.insert(dz.end(), dz_i.begin(), dz_i.end());
  std::vector<R> dw(dw_r);
  dw.insert(dw.end(), dw_i.begin(), dw_i.end());
  int rc;
  uint32_t *dgx, *dtz, *ddz;
  int32_t *dgoff, *dgmid, *dchunk, *dlchunk;
  uint8_t *dchunk_xl, *dlchunk_xl;
  uint64_t* dgbk;
  R *dtw, *ddw;
  HLut<R>* dhl = nullptr;
  if ((rc = upload(d, &dgx, gx, bytes)) || (rc = upload(d, &dgoff, goff, bytes)) ||
      (rc = upload(d, &dgmid, gmid, bytes)) || (rc = upload(d, &dchunk, chunk, bytes)) ||
      (rc = upload(d, &dchunk_xl, chunk_xl, bytes)) || (rc = upload(d, &dtz, tz, bytes)) ||
      (rc = upload(d, &dtw, tw, bytes)) || (rc = upload(d, &ddz, dz, bytes)) ||
      (rc = upload(d, &ddw, dw, bytes)) || (rc = upload(d, &dhl, hl, bytes)) ||
      (rc = upload(d, &dlchunk, lchunk, bytes)) || (rc = upload(d, &dlchunk_xl, lchunk_xl, bytes)) ||
      (rc = upload(d, &dgbk, gbk, bytes)))
    return rc;
  d.t.gbk = dgbk;
  d.t.n = p.n_qubits;
  d.t.G = G;
  d.t.T = (int64_t)tz.size();
  d.t.n_chunks = (int)chunk.size() - 1;
  d.t.gx = dgx;
  d.t.goff = dgoff;
  d.t.gmid = dgmid;
  d.t.chunk_g = dchunk;
  d.t.chunk_xl = dchunk_xl;
  d.t.tz = dtz;
  d.t.tw = dtw;
  d.t.nd = (int)dz.size();
  d.t.nd_mid = (int)dz_r.size();
  d.t.dz = ddz;
  d.t.dw = ddw;
  d.t.GL = (int)hl.size();
  d.t.hlut = dhl;
  d.t.n_lchunks = (int)lchunk.size() - 1;
  d.t.lchunk = dlchunk;
  d.t.lchunk_xl = dlchunk_xl;
  {
    // coupling bound for the scatter kernel's fixed-point scale
    double hb = std::fabs(ident), dm = 0.0;
    for (const HLut<R>& L : hl) {
      double m = 0.0;
      for (int c = 0; c < 16; ++c) m = std::max(m, std::fabs((double)L.lut16[c]));
      hb += m;
      dm = std::max(dm, m);
    }
    for (size_t g = 0; g + 1 < goff.size(); ++g) {
      double m = 0.0;
      for (int32_t t = goff[g]; t < goff[g + 1]; ++t) m += std::fabs((double)tw[t]);
      hb += m;
      dm = std::max(dm, m);
    }
    for (const R& w : dw) hb += std::fabs((double)w);
    d.t.hbound = hb;
    d.t.dmax = dm;
  }
  if ((rc = build_tiled<R>(p.n_qubits, hl, gx, goff, gmid, gbk, tz, tw, d, bytes))) return rc;
  // ---- pool
  const Pool& P = p.pool;
  const int M = P.size();
  std::vector<uint32_t> px(M), pz;
  std::vector<int32_t> poff, pmid(M), porder(M);
  std::vector<R> pw, pw2;
  for (int k = 0; k < M; ++k) {
    poff.push_back((int32_t)pz.size());
    px[k] = P.off[k + 1] > P.off[k] ? P.x[P.off[k]] : 0u;
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1) pmid[k] = (int32_t)pz.size();
      for (int64_t s = P.off[k]; s < P.off[k + 1]; ++s) {
        bool imag = false;
        double w = eff_weight(P.coeff[s], P.phase[s], P.x[s], P.z[s], &imag);
        if ((int)imag != pass) continue;
        pz.push_back(P.z[s]);
        pw.push_back((R)w);
        pw2.push_back((R)(parity32(px[k] & P.z[s]) ? -w : w));
      }
    }
  }
  poff.push_back((int32_t)pz.size());
  std::vector<LutDev<R>> pl(M);
  std::vector<PairEnum> pe(M);
  uint32_t pe_max = 0;
  bool all_lut = M > 0;
  for (int k = 0; k < M && all_lut; ++k) {
    std::vector<uint32_t> zz;
    std::vector<double> ww;
    for (int64_t s2 = P.off[k]; s2 < P.off[k + 1]; ++s2) {
      bool imag = false;
      double w = eff_weight(P.coeff[s2], P.phase[s2], P.x[s2], P.z[s2], &imag);
      if (imag) { all_lut = false; break; }
      zz.push_back(P.z[s2]);
      ww.push_back(w);
    }
    if (all_lut && !make_lut<R>(px[k], zz, ww, &pl[k])) all_lut = false;
    if (all_lut) {
      LutForm f = lut_form(zz.data(), ww.data(), (int)zz.size());
      if (!make_enum(f, px[k], p.n_qubits, &pe[k])) {
        // a generator that touches nothing: an empty enumeration
        std::memset(&pe[k], 0, sizeof(PairEnum));
      }
      pe_max = std::max(pe_max, (uint32_t)pe[k].ncodes << pe[k].log2cnt);
    }
  }
  for (int k = 0; k < M; ++k) porder[k] = k;
  std::stable_sort(porder.begin(), porder.end(), [&](int a, int b) {
    return P.family[a] < P.family[b];
  });
  uint32_t *dpx, *dpz;
  int32_t *dpoff, *dpmid, *dporder;
  R *dpw, *dpw2;
  if ((rc = upload(d, &dpx, px, bytes)) || (rc = upload(d, &dpoff, poff, bytes)) ||
      (rc = upload(d, &dpmid, pmid, bytes)) || (rc = upload(d, &dpz, pz, bytes)) ||
      (rc = upload(d, &dpw, pw, bytes)) || (rc = upload(d, &dpw2, pw2, bytes)) ||
      (rc = upload(d, &dporder, porder, bytes)))
    return rc;
  d.t.M = M;
  d.t.S = (int64_t)pz.size();
  d.t.px = dpx;
  d.t.poff = dpoff;
  d.t.pmid = dpmid;
  d.t.pz = dpz;
  d.t.pw = dpw;
  d.t.pw2 = dpw2;
  d.t.porder = dporder;
  if (all_lut) {
    LutDev<R>* dpl = nullptr;
    PairEnum* dpe;
    if ((rc = upload(d, &dpl, pl, bytes)) || (rc = upload(d, &dpe, pe, bytes))) return rc;
    d.t.plut = dpl;
    d.t.penum = dpe;
    d.t.penum_max = pe_max;
    d.t.pool_lut = true;
  }
  if (p.sector) {
    // ---- sector layout: occupation-space flips and paired term lists
    if (!all_lut && M > 0) return fail(GOCP_EINVAL, "sector layout needs generators in LUT form");
    const Encoding enc = make_encoding(p.mapping, p.n_qubits);
    auto flip = [&](uint32_t x) {
      const uint32_t u = enc.decode(x);
      uint32_t a = 0, b = 0;
      for (int q = 0; 2 * q < p.n_qubits; ++q) {
        a |= ((u >> (2 * q)) & 1u) << q;
        b |= ((u >> (2 * q + 1)) & 1u) << q;
      }
      return a | (b << 16);
    };
    std::vector<uint32_t> hu, gu, pu;
    for (const HLut<R>& L : hl) hu.push_back(flip(L.x));
    for (uint32_t x : gx) gu.push_back(flip(x));
    for (int k = 0; k < M; ++k) pu.push_back(flip(px[k]));
    std::vector<uint32_t> sdel, sneg, sz;
    std::vector<int32_t> soff, smid;
    std::vector<R> sw;
    for (int g = 0; g < G; ++g) {
      const auto pr = paired_terms<R>(tz, tw, goff[g], gmid[g], goff[g + 1]);
      soff.push_back((int32_t)sz.size());
      sdel.push_back(pr.delta);
      sneg.push_back(pr.neg);
      if (pr.delta) {
        sz.insert(sz.end(), pr.z.begin(), pr.z.end());
        sw.insert(sw.end(), pr.w.begin(), pr.w.end());
        smid.push_back((int32_t)sz.size());
      } else {
        for (int32_t t = goff[g]; t < gmid[g]; ++t) {
          sz.push_back(tz[t]);
          sw.push_back(tw[t]);
        }
        smid.push_back((int32_t)sz.size());
        for (int32_t t = gmid[g]; t < goff[g + 1]; ++t) {
          sz.push_back(tz[t]);
          sw.push_back(tw[t]);
        }
      }
    }
    soff.push_back((int32_t)sz.size());
    uint32_t *dhu, *dgu, *dpu, *dsdel, *dsneg, *dsz;
    int32_t *dsoff, *dsmid;
    R* dsw;
    if ((rc = upload(d, &dhu, hu, bytes)) || (rc = upload(d, &dgu, gu, bytes)) || (rc = upload(d, &dpu, pu, bytes)) ||
        (rc = upload(d, &dsdel, sdel, bytes)) || (rc = upload(d, &dsneg, sneg, bytes)) ||
        (rc = upload(d, &dsoff, soff, bytes)) || (rc = upload(d, &dsmid, smid, bytes)) ||
        (rc = upload(d, &dsz, sz, bytes)) || (rc = upload(d, &dsw, sw, bytes)))
      return rc;
    d.t.hu = dhu;
    d.t.gu = dgu;
    d.t.pu = dpu;
    d.t.sp_delta = dsdel;
    d.t.sp_neg = dsneg;
    d.t.sp_off = dsoff;
    d.t.sp_mid = dsmid;
    d.t.sp_z = dsz;
    d.t.sp_w = dsw;
  }
  return GOCP_OK;
}

int grid_for(uint64_t work, int sm_count, int per_sm) {
  uint64_t want = (work + kThreads - 1) / kThreads;
  uint64_t cap = (uint64_t)sm_count * per_sm;
  return (int)std::max<uint64_t>(1, std::min(want, cap));
}

int apply_grid(int n) { return (int)std::max<uint64_t>(1, ((1ull << n) + kTileH - 1) / kTileH); }
int pool_grid_x(const DeviceTables& d) { return grid_for(1ull << d.t.n, d.sm_count, 2); }
int pool_lut_nbx(uint32_t max_pairs) {
  const uint64_t per = (uint64_t)kThreads * kPairsPerThread;
  return (int)std::max<uint64_t>(1, (max_pairs + per - 1) / per);
}

}  // namespace

int upload_problem(Problem& p) {
  if (p.device < 0) return GOCP_OK;
  cudaError_t e = cudaSetDevice(p.device);
  if (e != cudaSuccess) return cuda_status(e, "cudaSetDevice");
  DeviceTables* d = new DeviceTables();
  p.dev = d;
  size_t bytes = 0;
  int rc;
  if (p.n_qubits >= 8) {
    const size_t words = (size_t)1 << (p.n_qubits - 8);
    const size_t blocks = (words + kThreads * kLiveWordsPerThread - 1) / (kThreads * kLiveWordsPerThread);
    if ((rc = dalloc(*d, &d->t.octmask, words, bytes)) || (rc = dalloc(*d, &d->t.octmask2, words, bytes)) ||
        (rc = dalloc(*d, &d->live.list, words * 32, bytes)) || (rc = dalloc(*d, &d->live.counts, blocks, bytes)) ||
        (rc = dalloc(*d, &d->live.len, 1, bytes)))
      return rc;
  }
  rc = p.precision == GOCP_C64 ? upload_typed<float>(p, *d, bytes, &p.identity)
                               : upload_typed<double>(p, *d, bytes, &p.identity);
  if (rc) return rc;
  if (p.n_qubits >= 8 && d->t.pool_lut) {
    // chain list: a quarter of the state's indices at most, one amplitude-mask bit each
    const int n = p.n_qubits;
    const size_t nb = ((((size_t)1 << (n - 5)) + 255) / 256) + 1;
    if ((rc = dalloc(*d, &d->t.cl.list, (size_t)1 << (n - 2), bytes)) ||
        (rc = dalloc(*d, &d->t.cl.amask, (size_t)1 << (n - 5), bytes)) || (rc = dalloc(*d, &d->t.cl.cnt, kRingWords, bytes)) ||
        (rc = dalloc(*d, &d->chain_counts, nb, bytes)))
      return rc;
    d->t.cl.cap = 1u << (n - 2);
  }
  int sm = 0;
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, p.device);
  d->sm_count = sm > 0 ? sm : 1;
  p.sm_count = d->sm_count;
  const int M = d->t.M;
  const int nchunks = (M + kOpsPerBlock - 1) / kOpsPerBlock;
  if (nchunks > kMaxChunks) return fail(GOCP_EINVAL, "pool too large for the gradient kernel");
  size_t need = 2 * (size_t)apply_grid(p.n_qubits);
  need = std::max(need, (size_t)pool_grid_x(*d) * (size_t)std::max(nchunks, 1) * kOpsPerBlock);
  need = std::max(need, (size_t)d->sm_count * 8);
  if (d->t.pool_lut)
    need = std::max(need, (size_t)std::max(nchunks, 1) * kOpsPerBlock * (size_t)pool_lut_nbx(d->t.penum_max));
  d->scratch_doubles = need;
  if ((rc = dalloc(*d, &d->scratch, need, bytes))) return rc;
  if ((rc = dalloc(*d, &d->counters, kMaxChunks + 8, bytes))) return rc;
  if ((rc = dalloc(*d, &d->scalars, 16, bytes))) return rc;
  if ((rc = dalloc(*d, &d->err, 1, bytes))) return rc;
  if ((rc = dalloc(*d, &d->selected, 1, bytes))) return rc;
  if ((rc = dalloc(*d, &d->grads, std::max(M, 1), bytes))) return rc;
  if ((rc = dalloc(*d, &d->graw, std::max(nchunks * kOpsPerBlock, 1), bytes))) return rc;
  cudaMemset(d->counters, 0, (kMaxChunks + 8) * sizeof(unsigned int));
  cudaMemset(d->err, 0, sizeof(int32_t));
  cudaMemset(d->scalars, 0, 16 * sizeof(double));
  p.device_bytes = bytes;
  return cuda_status(cudaDeviceSynchronize(), "upload");
}

void free_device(Problem& p) {
  if (!p.dev) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (p.device >= 0) cudaSetDevice(p.device);
  for (void* q : p.dev->allocs) cudaFree(q);
  if (cur >= 0) cudaSetDevice(cur);
  delete p.dev;
  p.dev = nullptr;
}

// Which on-chip chain forms may run: GOCP_ONCHIP_CHAINS = "all" (one block
// and clusters), "block" (one block only), "off" (the grid kernels only);
// default "block" for complex64 and "off" for complex128, whose FP64
// arithmetic is better spread over every SM than held in a few.
enum { kOnchipOff = 0, kOnchipBlock = 1, kOnchipAll = 2 };
int onchip_mode(int precision) {
  const char* e = std::getenv("GOCP_ONCHIP_CHAINS");
  if (e && *e) {
    if (!std::strcmp(e, "all")) return kOnchipAll;
    if (!std::strcmp(e, "block")) return kOnchipBlock;
    if (!std::strcmp(e, "off")) return kOnchipOff;
  }
  return precision == GOCP_C64 ? kOnchipBlock : kOnchipOff;
}

// ---- chains in cluster shared memory (DSMEM)
//
// A state too large for one block's shared memory but not for a cluster's
// (kClusterMax blocks x kSmemStateBytes: 2 MiB) is spread over the blocks of
// one thread-block cluster: block r holds amplitudes [r S, (r + 1) S), S =
// 2^n / C.  Each step splits the operator's enumerated touched pairs over
// the whole cluster; a thread reaches the two ends of its pair in whichever
// block holds them (distributed shared memory, through map_shared_rank) and
// computes them with the same per-pair arithmetic (taylor_pair_at,
// adjoint_pair_at), so the forward chain gives the same state bit for bit.
// A cluster barrier separates the steps.  The backward sweep keeps psi and
// lambda (two slices per block); each dE_j is the fixed-order sum of the
// blocks' partials, gathered in block 0.
constexpr int kClusterMax = 16;

template <typename R>
__device__ void taylor_chain_cluster_body(const DevTables& tb, const int32_t* ops, const double* coefs, int n_ops,
                                          C_t<R>* psi, int32_t* err, uint32_t* mask, uint8_t* cs_raw) {
  cg::cluster_group cl = cg::this_cluster();
  const uint32_t C = cl.num_blocks(), rank = cl.block_rank();
  const uint32_t dim = 1u << tb.n, slice = dim / C;
  const int shift = __ffs((int)slice) - 1;
  C_t<R>* mine = reinterpret_cast<C_t<R>*>(cs_raw);
  StepDesc<R>* sd = reinterpret_cast<StepDesc<R>*>(mine + slice);
  smem_copy_in<R>(mine, psi + (size_t)rank * slice, slice);
  cl.sync();
  for (int j = 0; j < n_ops; ++j) {
    if (j % kStepChunk == 0) stage_steps<R>(tb, ops, coefs, j, min(n_ops, j + kStepChunk), sd, err, rank == 0);
    const StepDesc<R>& D = sd[j % kStepChunk];
    if (!D.valid) continue;   // acts as the identity, flagged
    const LutDev<R>& L = D.L;
    const PairEnum& E = D.E;
    R c[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) c[m] = D.c[m];
    const uint32_t count = (uint32_t)E.ncodes << E.log2cnt;
    for (uint32_t q = rank * kSmemThreads + threadIdx.x; q < count; q += C * kSmemThreads) {
      uint32_t ph;
      const uint32_t b = enum_pair(E, q, &ph), b2 = b ^ L.x;
      C_t<R>* p1 = cl.map_shared_rank(mine + (b & (slice - 1u)), b >> shift);
      C_t<R>* p2 = cl.map_shared_rank(mine + (b2 & (slice - 1u)), b2 >> shift);
      if (cz<R>(*p1) && cz<R>(*p2)) continue;   // T maps (0, 0) to (0, 0)
      C_t<R> o1, o2;
      taylor_pair_at<R>(L, c, b, ph, p1, p2, o1, o2);
    }
    cl.sync();
  }
  smem_copy_out<R>(psi + (size_t)rank * slice, mine, slice);
  if (mask) {   // the exact nonzero-octet mask of this block's slice
    const uint32_t o_base = rank * (slice >> 3);
    for (uint32_t o0 = 0; o0 < ((slice + 7u) >> 3); o0 += kSmemThreads) {
      const uint32_t o = o0 + threadIdx.x;
      bool nz = false;
      if (o < (slice >> 3))
        for (int i = 0; i < 8; ++i) nz |= mine[8u * o + i].x != R(0) || mine[8u * o + i].y != R(0);
      const uint32_t word = __ballot_sync(0xffffffffu, nz);
      if ((threadIdx.x & 31) == 0 && o < (slice >> 3)) mask[(o_base + o) >> 5] = word;
    }
  }
  cl.sync();   // no block leaves while another may still read its shared memory
}

template <typename R>
__global__ void __launch_bounds__(kSmemThreads, 1)
k_taylor_chain_cluster(DevTables tb, const int32_t* ops, const double* coefs, int n_ops, C_t<R>* psi,
                       int32_t* err, uint32_t* mask) {
  extern __shared__ __align__(16) uint8_t cs_raw[];
  taylor_chain_cluster_body<R>(tb, ops, coefs, n_ops, psi, err, mask, cs_raw);
}

template <typename R>
__device__ void adjoint_chain_cluster_body(const DevTables& tb, const int32_t* ops, const double* coefs, int n_ops,
                                           C_t<R>* psi, C_t<R>* lam, double* dtheta, int32_t* err,
                                           uint8_t* cs_raw) {
  __shared__ double s_red[kSmemThreads / 32];
  __shared__ double s_part[kClusterMax];   // block 0's: the blocks' partials of dE_j
  cg::cluster_group cl = cg::this_cluster();
  const uint32_t C = cl.num_blocks(), rank = cl.block_rank();
  const uint32_t dim = 1u << tb.n, slice = dim / C;
  const int shift = __ffs((int)slice) - 1;
  C_t<R>* mp = reinterpret_cast<C_t<R>*>(cs_raw);
  C_t<R>* ml = mp + slice;
  StepDesc<R>* sd = reinterpret_cast<StepDesc<R>*>(ml + slice);
  smem_copy_in<R>(mp, psi + (size_t)rank * slice, slice);
  smem_copy_in<R>(ml, lam + (size_t)rank * slice, slice);
  double* part0 = cl.map_shared_rank(s_part, 0u);
  cl.sync();
  for (int j = n_ops - 1; j >= 0; --j) {
    const int jc = j - j % kStepChunk;
    if (j == n_ops - 1 || j % kStepChunk == kStepChunk - 1)
      stage_steps<R>(tb, ops, coefs, jc, min(n_ops, jc + kStepChunk), sd, err, rank == 0);
    const StepDesc<R>& D = sd[j - jc];
    if (!D.valid) {
      if (rank == 0 && threadIdx.x == 0) dtheta[j] = 0.0;
      continue;
    }
    const LutDev<R>& L = D.L;
    const PairEnum& E = D.E;
    R c[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) c[m] = D.c[m];
    const uint32_t count = (uint32_t)E.ncodes << E.log2cnt;
    double v = 0.0;
    for (uint32_t q = rank * kSmemThreads + threadIdx.x; q < count; q += C * kSmemThreads) {
      uint32_t ph;
      const uint32_t b = enum_pair(E, q, &ph), b2 = b ^ L.x;
      const uint32_t r1 = b >> shift, r2 = b2 >> shift, o1 = b & (slice - 1u), o2 = b2 & (slice - 1u);
      C_t<R>* a1 = cl.map_shared_rank(mp + o1, r1);
      C_t<R>* a2 = cl.map_shared_rank(mp + o2, r2);
      C_t<R>* l1 = cl.map_shared_rank(ml + o1, r1);
      C_t<R>* l2 = cl.map_shared_rank(ml + o2, r2);
      if (cz<R>(*a1) && cz<R>(*a2) && cz<R>(*l1) && cz<R>(*l2)) continue;   // nothing to add, stays zero
      C_t<R> o[4];
      v += adjoint_pair_at<R>(L, c, b, ph, a1, a2, l1, l2, o);
    }
    const double w = __any_sync(0xffffffffu, v != 0.0) ? warp_sum(v) : 0.0;
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < kSmemThreads / 32; ++q) t += s_red[q];
      part0[rank] = t;
    }
    cl.sync();   // every pair of step j done, every partial in block 0
    if (rank == 0 && threadIdx.x == 0) {
      double t = 0.0;
      for (uint32_t r = 0; r < C; ++r) t += s_part[r];
      dtheta[j] = t;
    }
    cl.sync();   // block 0 has read the partials before the next step writes them
  }
  smem_copy_out<R>(psi + (size_t)rank * slice, mp, slice);
  smem_copy_out<R>(lam + (size_t)rank * slice, ml, slice);
  cl.sync();
}

template <typename R>
__global__ void __launch_bounds__(kSmemThreads, 1)
k_adjoint_chain_cluster(DevTables tb, const int32_t* ops, const double* coefs, int n_ops, C_t<R>* psi,
                        C_t<R>* lam, double* dtheta, int32_t* err) {
  extern __shared__ __align__(16) uint8_t cs_raw[];
  adjoint_chain_cluster_body<R>(tb, ops, coefs, n_ops, psi, lam, dtheta, err, cs_raw);
}

// The same for items whose state(s) need a cluster: one cluster per item,
// items[first + blockIdx.x / cluster size].
template <typename R>
__global__ void __launch_bounds__(kSmemThreads, 1) k_stage_forward_cluster(const BatchItemDev* items, int first) {
  extern __shared__ __align__(16) uint8_t cs_raw[];
  const BatchItemDev& it = items[first + blockIdx.x / cg::this_cluster().num_blocks()];
  taylor_chain_cluster_body<R>(it.t, it.ops, it.coefs, it.n_ops, (C_t<R>*)it.psi, it.err, nullptr, cs_raw);
}

template <typename R>
__global__ void __launch_bounds__(kSmemThreads, 1) k_stage_backward_cluster(const BatchItemDev* items, int first) {
  extern __shared__ __align__(16) uint8_t cs_raw[];
  const BatchItemDev& it = items[first + blockIdx.x / cg::this_cluster().num_blocks()];
  adjoint_chain_cluster_body<R>(it.t, it.ops, it.coefs, it.n_ops, (C_t<R>*)it.psi, (C_t<R>*)it.lam, it.dtheta,
                                it.err, cs_raw);
}

// Blocks of the cluster that holds `states` states of this problem in
// shared memory (a power of two, 2 .. kClusterMax), or 0 when one block
// does or none fits.
template <typename R>
int chain_cluster_blocks(const DeviceTables& d, int states) {
  if (!d.t.pool_lut || onchip_mode(sizeof(R) == 4 ? GOCP_C64 : GOCP_C128) < kOnchipAll) return 0;
  const uint64_t bytes = ((uint64_t)states << d.t.n) * sizeof(C_t<R>);
  if (bytes <= kSmemStateBytes) return 0;
  for (int c = 2; c <= kClusterMax; c *= 2)
    if (bytes <= (uint64_t)c * kSmemStateBytes && (1ull << d.t.n) % (uint64_t)c == 0) return c;
  return 0;
}

// Whether one cluster of `blocks` blocks of `kernel` (kSmemThreads threads,
// bytes of dynamic shared memory each) can be resident on this device.
bool cluster_fits_query(const void* kernel, int blocks, size_t bytes) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks, 1, 1);
  cfg.blockDim = dim3(kSmemThreads, 1, 1);
  cfg.dynamicSmemBytes = bytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)blocks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return clusters > 0;
}

// cluster_fits_query, remembered per (device, kernel, blocks, bytes).
bool cluster_fits(const void* kernel, int blocks, size_t bytes) {
  struct Key {
    int device;
    const void* kernel;
    int blocks;
    size_t bytes;
  };
  static std::mutex mu;
  static std::vector<std::pair<Key, bool>> seen;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> lk(mu);
  for (const auto& e : seen)
    if (e.first.device == device && e.first.kernel == kernel && e.first.blocks == blocks && e.first.bytes == bytes)
      return e.second;
  const bool ok = cluster_fits_query(kernel, blocks, bytes);
  seen.push_back({Key{device, kernel, blocks, bytes}, ok});
  return ok;
}

// Launches `kernel` as `clusters` clusters of `blocks` blocks (kSmemThreads
// each, bytes of dynamic shared memory each).
int launch_cluster(const void* kernel, int blocks, size_t bytes, void** args, cudaStream_t st, int clusters = 1) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(blocks * clusters), 1, 1);
  cfg.blockDim = dim3(kSmemThreads, 1, 1);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)blocks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cuda_status(cudaLaunchKernelExC(&cfg, kernel, args), "cluster chain launch");
}

// Whether the on-chip forward chain / backward sweep takes this problem.
template <typename R>
bool smem_chain_fits(const DeviceTables& d, int states) {
  return d.t.pool_lut && onchip_mode(sizeof(R) == 4 ? GOCP_C64 : GOCP_C128) >= kOnchipBlock &&
         ((uint64_t)states << d.t.n) * sizeof(C_t<R>) <= kSmemStateBytes;
}

// Opts the on-chip chain kernels into kSmemStateBytes of dynamic shared
// memory on the current device (once per device).
template <typename R>
int smem_chain_optin() {
  static std::mutex mu;
  static std::vector<bool> done;
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(mu);
  if (device >= (int)done.size()) done.resize(device + 1, false);
  if (!done[device]) {
    e = cudaFuncSetAttribute(k_taylor_chain_smem<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSmemStateBytes + kSmemDescBytes));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_adjoint_chain_smem<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kSmemStateBytes + kSmemDescBytes));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_stage_forward_all<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kSmemStateBytes + kSmemDescBytes));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_stage_backward_all<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kSmemStateBytes + kSmemDescBytes));
    for (const void* k : {(const void*)k_taylor_chain_cluster<R>, (const void*)k_adjoint_chain_cluster<R>,
                          (const void*)k_stage_forward_cluster<R>, (const void*)k_stage_backward_cluster<R>}) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kSmemStateBytes + kSmemDescBytes));
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
    if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(on-chip chains)");
    done[device] = true;
  }
  return GOCP_OK;
}

// ------------------------------------------------------------ launchers

// Blocks of an adjoint step (k_adjoint).
int adjoint_grid(const DeviceTables& d) {
  if (d.t.pool_lut) return grid_for((uint64_t)d.t.penum_max, d.sm_count, kChainBlocksPerSm);
  return grid_for(1ull << (d.t.n - 1), d.sm_count, 8);
}

int ensure_stage(Problem& p, int n_ops) {
  DeviceTables& d = *p.dev;
  if (n_ops <= d.stage_cap) return GOCP_OK;
  int cap = std::max(n_ops, 2 * d.stage_cap);
  cap = std::max(cap, 256);
  size_t bytes = 0;
  int rc;
  // earlier staging buffers stay allocated until the problem is freed, so
  // work still queued on a stream never sees them disappear
  if ((rc = dalloc(d, &d.stage_ops, cap, bytes)) || (rc = dalloc(d, &d.stage_theta, cap, bytes)) ||
      (rc = dalloc(d, &d.coefs, (size_t)cap * 6, bytes)) || (rc = dalloc(d, &d.dtheta, cap, bytes)))
    return rc;
  // per-block partials of the adjoint sweep (LUT pools): one row of blocks per op
  if (d.t.pool_lut && (rc = dalloc(d, &d.dpart, (size_t)cap * adjoint_grid(d), bytes))) return rc;
  p.device_bytes += bytes;
  d.stage_cap = cap;
  return GOCP_OK;
}

int32_t* stage_ops_ptr(Problem& p) { return p.dev->stage_ops; }
double* stage_theta_ptr(Problem& p) { return p.dev->stage_theta; }
double* dtheta_ptr(Problem& p) { return p.dev->dtheta; }
double* scalars_ptr(Problem& p) { return p.dev->scalars; }
double* grads_ptr(Problem& p) { return p.dev->grads; }
int32_t* selected_ptr(Problem& p) { return p.dev->selected; }
int32_t* err_ptr(Problem& p) { return p.dev->err; }
// ------------------------------------------------------------ launch chains

struct ChainCache {
  struct Entry {
    std::string key;
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;
  };
  std::vector<Entry> entries;
  uint64_t clock = 0;
};
constexpr size_t kChainCacheSize = 8;

void free_chains(Problem& p) {
  if (!p.chains) return;
  for (auto& e : p.chains->entries)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  delete p.chains;
  p.chains = nullptr;
}

namespace {

// n plain launches (when a graph cannot be made)
int launch_plain(const void* kernel, unsigned grid, unsigned block, int n, bool reverse, void** args, int jidx,
                 cudaStream_t st) {
  int& j = *static_cast<int*>(args[jidx]);
  for (int i = 0; i < n; ++i) {
    j = reverse ? n - 1 - i : i;
    cudaError_t e = cudaLaunchKernel(kernel, dim3(grid), dim3(block), args, 0, st);
    if (e != cudaSuccess) return cuda_status(e, "chain launch");
  }
  return GOCP_OK;
}

}  // namespace

// Whether consecutive steps of a chain graph are joined by programmatic
// edges (GOCP_CHAIN_PDL=0 joins them by full completion instead).  Every
// kernel passed to launch_chain starts with chain_step_begin(), so step j + 1
// reads nothing before step j has finished either way; the programmatic edge
// only lets its blocks be scheduled earlier.
bool chain_pdl() {
  const char* e = std::getenv("GOCP_CHAIN_PDL");
  return !(e && !std::strcmp(e, "0"));
}

int launch_chain(Problem& p, const void* kernel, unsigned grid, unsigned block, int n, bool reverse, void** args,
                 const size_t* sizes, int nargs, int jidx, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (n <= 0) return GOCP_OK;
  count_launches(n);
  const bool pdl = chain_pdl();
  std::string key((const char*)&kernel, sizeof(kernel));
  const unsigned hdr[5] = {grid, block, (unsigned)n, reverse ? 1u : 0u, pdl ? 1u : 0u};
  key.append((const char*)hdr, sizeof(hdr));
  for (int i = 0; i < nargs; ++i)
    if (i != jidx) key.append((const char*)args[i], sizes[i]);
  if (!p.chains) p.chains = new ChainCache();
  ChainCache& c = *p.chains;
  ++c.clock;
  for (auto& e : c.entries)
    if (e.key == key) {
      e.used = c.clock;
      return cuda_status(cudaGraphLaunch(e.exec, st), "chain graph launch");
    }
  // build the graph: n kernel nodes in a line, node i with op index j(i),
  // each depending on the one before (programmatically where possible)
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) {
    cudaGetLastError();
    return launch_plain(kernel, grid, block, n, reverse, args, jidx, st);
  }
  int& j = *static_cast<int*>(args[jidx]);
  const int j_saved = j;
  cudaGraphNode_t prev = nullptr;
  bool ok = true;
  for (int i = 0; i < n && ok; ++i) {
    j = reverse ? n - 1 - i : i;
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(kernel);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.kernelParams = args;
    cudaGraphNode_t node;
    ok = cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp) == cudaSuccess;
    if (ok && prev) {
      cudaGraphEdgeData ed = {};
      ed.from_port = cudaGraphKernelNodePortProgrammatic;
      ed.type = cudaGraphDependencyTypeProgrammatic;
      if (!pdl || cudaGraphAddDependencies(g, &prev, &node, &ed, 1) != cudaSuccess) {
        cudaGetLastError();
        ok = cudaGraphAddDependencies(g, &prev, &node, nullptr, 1) == cudaSuccess;
      }
    }
    prev = node;
  }
  j = j_saved;
  cudaGraphExec_t exec = nullptr;
  if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    return launch_plain(kernel, grid, block, n, reverse, args, jidx, st);
  }
  if (c.entries.size() >= kChainCacheSize) {
    auto lru = std::min_element(c.entries.begin(), c.entries.end(),
                                [](const ChainCache::Entry& a, const ChainCache::Entry& b) { return a.used < b.used; });
    cudaGraphExecDestroy(lru->exec);
    c.entries.erase(lru);
  }
  c.entries.push_back({key, exec, c.clock});
  return cuda_status(cudaGraphLaunch(exec, st), "chain graph launch");
}

// for the sector-layout launchers (sector.cu)
const DevTables& dev_tables(Problem& p) { return p.dev->t; }
double* coefs_ptr(Problem& p) { return p.dev->coefs; }
double* scratch_ptr(Problem& p, size_t* doubles) {
  *doubles = p.dev->scratch_doubles;
  return p.dev->scratch;
}
unsigned int* counters_ptr(Problem& p) { return p.dev->counters + kMaxChunks; }   // 8 slots, zero at rest

// Pool gradients from block partials part[i * nbx + b] (i in GOCP family
// order): grads[porder[i]] = 2 sum_b part[i nbx + b] / <psi|psi> (scalars[1]).
int pool_finish(Problem& p, const double* part, int nbx, double* d_grads, cudaStream_t st) {
  DeviceTables& d = *p.dev;
  const int M = d.t.M;
  if (M == 0) return GOCP_OK;
  k_pool_reduce<<<(M + 7) / 8, 256, 0, st>>>(part, nbx, M, d.graw);
  k_grad_final<<<(M + 255) / 256, 256, 0, st>>>(d.graw, d.t.porder, M, d.scalars, d_grads);
  count_launches(2);
  return cuda_status(cudaGetLastError(), "pool gradient reduction");
}

template <typename R>
static int launch_setup(Problem& p, void* psi, const double* d_theta, int n_ops, cudaStream_t st) {
  const uint64_t dim = psi ? 1ull << p.n_qubits : 1;
  int grid = grid_for(dim, p.dev->sm_count, 8);
  k_setup<R><<<grid, kThreads, 0, st>>>((C_t<R>*)psi, p.n_qubits, p.ref_index, d_theta, n_ops,
                                        p.dev->coefs, psi ? p.dev->t.octmask : nullptr, p.dev->t.cl);
  count_launches(1);
  return cuda_status(cudaGetLastError(), "k_setup");
}

// psi = |ref> (skipped when psi is NULL) and the Taylor coefficients of the
// staged ansatz (n_ops may be 0).  With psi, the problem's octet mask then
// describes psi (see dev_taylor_chain).
int dev_setup(Problem& p, void* psi, const double* d_theta, int n_ops, cudaStream_t st) {
  int rc = ensure_stage(p, n_ops);
  if (rc) return rc;
  return p.precision == GOCP_C64 ? launch_setup<float>(p, psi, d_theta, n_ops, st)
                                 : launch_setup<double>(p, psi, d_theta, n_ops, st);
}

template <typename R>
static int launch_taylor_chain(Problem& p, const int32_t* d_ops, int n_ops, void* psi, bool tracked,
                               cudaStream_t st) {
  DeviceTables& d = *p.dev;
  // chains of several steps on chip (a single step gains nothing from
  // loading and storing the whole state, and stays on the grid kernels)
  if (n_ops > 1 && smem_chain_fits<R>(d, 1)) {   // the whole chain in one block
    int rc = smem_chain_optin<R>();
    if (rc) return rc;
    ProfScope ps(GOCP_KERNEL_TAYLOR, st, 1);
    k_taylor_chain_smem<R><<<1, kSmemThreads, ((size_t)sizeof(C_t<R>) << p.n_qubits) + kSmemDescBytes, st>>>(
        d.t, d_ops, d.coefs, n_ops, (C_t<R>*)psi, d.err, tracked ? d.t.octmask : nullptr);
    count_launches(1);
    return cuda_status(cudaGetLastError(), "k_taylor_chain_smem");
  }
  if (n_ops > 1) {   // the whole chain in one cluster's shared memory
    const int cb = chain_cluster_blocks<R>(d, 1);
    int rc = cb > 0 ? smem_chain_optin<R>() : GOCP_OK;
    if (rc) return rc;
    const size_t bytes = cb > 0 ? ((sizeof(C_t<R>) << p.n_qubits) / cb + kSmemDescBytes) : 0;
    if (cb > 0 && cluster_fits((const void*)k_taylor_chain_cluster<R>, cb, bytes)) {
      DevTables tb = d.t;
      const int32_t* ops_ = d_ops;
      const double* coefs = d.coefs;
      int n = n_ops;
      C_t<R>* ps_ = (C_t<R>*)psi;
      int32_t* err = d.err;
      uint32_t* mk = tracked ? d.t.octmask : nullptr;
      void* args[] = {&tb, &ops_, &coefs, &n, &ps_, &err, &mk};
      ProfScope ps(GOCP_KERNEL_TAYLOR, st, 1);
      rc = launch_cluster((const void*)k_taylor_chain_cluster<R>, cb, bytes, args, st);
      count_launches(1);
      return rc;
    }
  }
  const int grid = d.t.pool_lut ? grid_for((uint64_t)d.t.penum_max, d.sm_count, kChainBlocksPerSm)
                                : grid_for(1ull << (p.n_qubits - 1), d.sm_count, 8);
  uint32_t* mask = tracked && d.t.pool_lut ? d.t.octmask : nullptr;
  DevTables tb = d.t;
  const double* coefs = d.coefs;
  int j = 0;
  C_t<R>* ps_ = (C_t<R>*)psi;
  int32_t* err = d.err;
  void* args[] = {&tb, &d_ops, &coefs, &j, &ps_, &err, &mask};
  // tb is fixed for the problem's lifetime (and the cache is the problem's): not part of the key
  const size_t sizes[] = {0, sizeof(d_ops), sizeof(coefs), sizeof(j), sizeof(ps_), sizeof(err), sizeof(mask)};
  ProfScope ps(GOCP_KERNEL_TAYLOR, st, n_ops);
  int rc = launch_chain(p, (const void*)k_taylor5<R>, grid, kThreads, n_ops, false, args, sizes, 7, 3, st);
  if (rc) return rc;
  return cuda_status(cudaGetLastError(), "k_taylor5");
}

// Applies operators 0..n_ops-1 of a staged ansatz whose coefficients were
// written by dev_setup.  `tracked`: psi is the state dev_setup just wrote
// (and the chain before it advanced), so the octet mask describes it; the
// chain then skips all-zero pairs and keeps the mask valid.
int dev_taylor_chain(Problem& p, const int32_t* d_ops, int n_ops, void* psi, bool tracked, cudaStream_t st) {
  if (n_ops == 0) return GOCP_OK;
  return p.precision == GOCP_C64 ? launch_taylor_chain<float>(p, d_ops, n_ops, psi, tracked, st)
                                 : launch_taylor_chain<double>(p, d_ops, n_ops, psi, tracked, st);
}

template <typename R>
static int launch_apply(Problem& p, const void* psi, void* hpsi, bool energy, cudaStream_t st) {
  DeviceTables& d = *p.dev;
  if (d.t.n_pieces > 0) {
    ProfScope ps(GOCP_KERNEL_APPLY_H, st);
    return tiled_apply_h(d.t, d.live, p.precision, d.sm_count, psi, hpsi, p.identity, energy ? d.scratch : nullptr,
                         d.counters + kMaxChunks, d.counters + kMaxChunks + 3, d.scalars, d.err, st);
  }
  const int grid = apply_grid(p.n_qubits);
  {
    ProfScope ps(GOCP_KERNEL_APPLY_H, st);
    k_apply_h<R><<<grid, kThreads, 0, st>>>(d.t, (const C_t<R>*)psi, (C_t<R>*)hpsi, p.identity,
                                            energy ? d.scratch : nullptr, d.counters + kMaxChunks,
                                            d.scalars);
  }
  count_launches(1);
  return cuda_status(cudaGetLastError(), "k_apply_h");
}

int dev_apply_h(Problem& p, const void* psi, void* hpsi, bool energy, cudaStream_t st) {
  return p.precision == GOCP_C64 ? launch_apply<float>(p, psi, hpsi, energy, st)
                                 : launch_apply<double>(p, psi, hpsi, energy, st);
}

template <typename R>
static int launch_norm(Problem& p, const void* psi, cudaStream_t st) {
  DeviceTables& d = *p.dev;
  const uint64_t dim = p.sector ? (uint64_t)p.sector_dim : 1ull << p.n_qubits;   // amplitudes of one state
  const int grid = grid_for(dim, d.sm_count, 8);
  k_norm<R><<<grid, kThreads, 0, st>>>((const C_t<R>*)psi, dim, d.scratch, d.counters + kMaxChunks + 1,
                                       d.scalars + 1);
  count_launches(1);
  return cuda_status(cudaGetLastError(), "k_norm");
}

int dev_norm(Problem& p, const void* psi, cudaStream_t st) {
  return p.precision == GOCP_C64 ? launch_norm<float>(p, psi, st) : launch_norm<double>(p, psi, st);
}

template <typename R>
static int launch_pool_grads(Problem& p, const void* psi, const void* hpsi, double* d_grads, bool mask_current,
                             cudaStream_t st) {
  DeviceTables& d = *p.dev;
  const int M = d.t.M;
  if (M == 0) return GOCP_OK;
  const int nchunks = (M + kOpsPerBlock - 1) / kOpsPerBlock;
  int n = 2;
  if (d.t.pool_lut) {
    const int nbx = pool_lut_nbx(d.t.penum_max);
    dim3 grid(nbx, nchunks);
    const uint32_t* mask = d.t.octmask;
    int rc;
    if (mask && !mask_current &&
        (rc = octet_mask(p.precision, psi, nullptr, p.n_qubits, d.t.octmask, nullptr, d.sm_count, st)))
      return rc;
    if (mask) {
      // the nonzero amplitudes of psi, one pass over them (k_pool_grad_amp);
      // when they do not fit the list (or the problem has none), the live
      // octets in index order and one pass over those (k_pool_grad_live)
      const bool amps = d.live.aidx != nullptr;
      const uint64_t octets = 1ull << (p.n_qubits - 3);
      int lnbx = (int)std::max<uint64_t>(1, std::min<uint64_t>(64, (octets + kThreads * 64 - 1) / (kThreads * 64)));
      lnbx = std::max(1, std::min<int>(lnbx, (int)(d.scratch_doubles / ((size_t)nchunks * kOpsPerBlock))));
      if (amps && (rc = amp_list(p.precision, psi, mask, p.n_qubits, d.live, st))) return rc;
      if ((rc = live_octets(mask, p.n_qubits, d.live, st))) return rc;
      {
        ProfScope ps(GOCP_KERNEL_POOL_GRAD, st, amps ? 2 : 1);
        if (amps)
          k_pool_grad_amp<R><<<dim3(lnbx, nchunks), kThreads, 0, st>>>(
              d.t, (const C_t<R>*)hpsi, d.live.aidx, (const C_t<R>*)d.live.aval, d.live.alen, d.live.acap,
              d.scratch, lnbx);
        k_pool_grad_live<R><<<dim3(lnbx, nchunks), kThreads, 0, st>>>(
            d.t, (const C_t<R>*)psi, (const C_t<R>*)hpsi, mask, d.live.list, d.live.len, d.scratch, lnbx,
            amps ? d.live.alen : nullptr, d.live.acap);
      }
      if (amps) ++n;
      k_pool_reduce<<<(M + 7) / 8, 256, 0, st>>>(d.scratch, lnbx, M, d.graw);
      ++n;
    } else {
      {
        ProfScope ps(GOCP_KERNEL_POOL_GRAD, st);
        k_pool_grad_lut<R><<<grid, kThreads, 0, st>>>(d.t, (const C_t<R>*)psi, (const C_t<R>*)hpsi,
                                                      d.scratch, nbx, mask);
      }
      k_pool_reduce<<<(M + 7) / 8, 256, 0, st>>>(d.scratch, nbx, M, d.graw);
      ++n;
    }
  } else {
    dim3 grid(pool_grid_x(d), nchunks);
    ProfScope ps(GOCP_KERNEL_POOL_GRAD, st);
    k_pool_grad<R><<<grid, kThreads, 0, st>>>(d.t, (const C_t<R>*)psi, (const C_t<R>*)hpsi,
                                              d.scratch, d.counters, d.graw);
  }
  k_grad_final<<<(M + 255) / 256, 256, 0, st>>>(d.graw, d.t.porder, M, d.scalars, d_grads);
  count_launches(n);
  return cuda_status(cudaGetLastError(), "k_pool_grad");
}

// `mask_current`: the problem's octet mask already describes psi (a tracked
// chain produced it); otherwise it is rebuilt from psi first.
// `norm_current`: scalars[1] already holds <psi|psi> (the energy epilogue of
// the H psi call just made on psi wrote it); otherwise k_norm computes it.
int dev_pool_grads(Problem& p, const void* psi, const void* hpsi, double* d_grads, bool mask_current,
                   bool norm_current, cudaStream_t st) {
  if (!norm_current) {
    int rc = dev_norm(p, psi, st);   // <psi|psi> -> scalars[1]
    if (rc) return rc;
  }
  return p.precision == GOCP_C64 ? launch_pool_grads<float>(p, psi, hpsi, d_grads, mask_current, st)
                                 : launch_pool_grads<double>(p, psi, hpsi, d_grads, mask_current, st);
}

template <typename R>
static int launch_adjoint(Problem& p, const int32_t* d_ops, int n_ops, void* psi, void* lam,
                          double* d_dE, cudaStream_t st) {
  DeviceTables& d = *p.dev;
  const uint64_t dim = 1ull << p.n_qubits;
  const int g1 = grid_for(dim, d.sm_count, 8);
  k_residual<R><<<g1, kThreads, 0, st>>>((const C_t<R>*)psi, (C_t<R>*)lam, p.n_qubits, d.scalars);
  if (smem_chain_fits<R>(d, 2)) {   // the whole sweep in one block
    count_launches(1);   // k_residual
    int rc = smem_chain_optin<R>();
    if (rc) return rc;
    ProfScope ps(GOCP_KERNEL_ADJOINT, st, 1);
    k_adjoint_chain_smem<R><<<1, kSmemThreads, ((size_t)(2 * sizeof(C_t<R>)) << p.n_qubits) + kSmemDescBytes,
                              st>>>(
        d.t, d_ops, d.coefs, n_ops, (C_t<R>*)psi, (C_t<R>*)lam, d_dE, d.err);
    count_launches(1);
    return cuda_status(cudaGetLastError(), "k_adjoint_chain_smem");
  }
  {
    const int cb = chain_cluster_blocks<R>(d, 2);
    int rc = cb > 0 ? smem_chain_optin<R>() : GOCP_OK;
    if (rc) return rc;
    const size_t bytes = cb > 0 ? ((2 * sizeof(C_t<R>) << p.n_qubits) / cb + kSmemDescBytes) : 0;
    if (cb > 0 && cluster_fits((const void*)k_adjoint_chain_cluster<R>, cb, bytes)) {   // the whole sweep in one cluster
      count_launches(1);   // k_residual
      DevTables tb = d.t;
      const double* coefs = d.coefs;
      int n = n_ops;
      C_t<R>* ps_ = (C_t<R>*)psi;
      C_t<R>* ls_ = (C_t<R>*)lam;
      int32_t* err = d.err;
      void* args[] = {&tb, &d_ops, &coefs, &n, &ps_, &ls_, &d_dE, &err};
      ProfScope ps(GOCP_KERNEL_ADJOINT, st, 1);
      rc = launch_cluster((const void*)k_adjoint_chain_cluster<R>, cb, bytes, args, st);
      count_launches(1);
      return rc;
    }
  }
  const int grid = adjoint_grid(d);
  // nonzero octets of psi or lambda, kept valid by the sweep
  uint32_t* mask = d.t.pool_lut ? d.t.octmask2 : nullptr;
  int rc;
  if (mask && (rc = octet_mask(p.precision, psi, lam, p.n_qubits, mask, nullptr, d.sm_count, st))) return rc;
  // the amplitudes nonzero in psi or lambda, kept complete by the sweep; its
  // first step, j = n_ops - 1, reads slot n_ops mod 3 and appends in slot
  // (n_ops - 1) mod 3
  if (mask && d.t.cl.list &&
      (rc = chain_list(p.precision, psi, lam, mask, p.n_qubits, d.t.cl, d.chain_counts, n_ops % 3,
                       (n_ops - 1) % 3, st)))
    return rc;
  double* dpart = d.t.pool_lut ? d.dpart : nullptr;
  count_launches(1);   // k_residual (and k_octet_mask counts itself)
  DevTables tb = d.t;
  const double* coefs = d.coefs;
  int j = 0;
  C_t<R>* ps_ = (C_t<R>*)psi;
  C_t<R>* ls_ = (C_t<R>*)lam;
  double* partials = d.scratch;
  unsigned int* counter = d.counters + kMaxChunks + 2;
  int32_t* err = d.err;
  void* args[] = {&tb, &d_ops, &coefs, &j, &ps_, &ls_, &partials, &counter, &d_dE, &err, &mask, &dpart};
  const size_t sizes[] = {0,           sizeof(d_ops),   sizeof(coefs), sizeof(j),    sizeof(ps_),  sizeof(ls_),
                          sizeof(partials), sizeof(counter), sizeof(d_dE), sizeof(err), sizeof(mask), sizeof(dpart)};
  ProfScope ps(GOCP_KERNEL_ADJOINT, st, n_ops + (dpart ? 1 : 0));
  if ((rc = launch_chain(p, (const void*)k_adjoint<R>, grid, kThreads, n_ops, true, args, sizes, 12, 3, st)))
    return rc;
  if (dpart) {
    k_dtheta_reduce<<<n_ops, kThreads, 0, st>>>(dpart, grid, d_dE);
    count_launches(1);
  }
  return cuda_status(cudaGetLastError(), "k_adjoint");
}

int dev_adjoint(Problem& p, const int32_t* d_ops, int n_ops, void* psi, void* lam, double* d_dE,
                cudaStream_t st) {
  return p.precision == GOCP_C64 ? launch_adjoint<float>(p, d_ops, n_ops, psi, lam, d_dE, st)
                                 : launch_adjoint<double>(p, d_ops, n_ops, psi, lam, d_dE, st);
}

int dev_select(Problem& p, const double* d_grads, double tie_rel, int32_t* d_out, cudaStream_t st) {
  k_select<<<1, kThreads, 0, st>>>(d_grads, p.dev->t.M, tie_rel, d_out);
  count_launches(1);
  return cuda_status(cudaGetLastError(), "k_select");
}


// ------------------------------------------------------------ allocation-free energy
//
// gocp_energy_static: H psi and the energy with the reduction scratch in a
// file-scope device array instead of the problem's allocated scratch.  For
// callers that cannot allocate device memory at the point of the call (a
// real-time or embedded host loop that must not block on cudaMalloc, a
// caller whose memory is owned by another allocator, work recorded between
// allocation-free checkpoints).  The problem's tables, the states and the
// outputs are still the caller's inputs and outputs.
//
// The array is shared by every call in the process: calls that overlap on
// the GPU race on it.  Every GPU that loads this library holds it (128 KiB
// of partials plus a few scalars) until the process exits.  Its device
// address is resolved once per device and kept; a cudaDeviceReset (or
// anything else that destroys the device's primary context) leaves that
// address stale, so no call may follow one in the same process.
//
// The H psi kernel is the untiled k_apply_h, the one gocp_energy runs below
// the tile size (13 qubits for complex64, 12 for complex128), with the same
// block decomposition there; from the tile size on gocp_energy runs the
// tiled kernels, which sum in another order.

constexpr int kStaticEnergyBlocks = 8192;   // one block per 2048-amplitude tile: n <= 24

struct StaticEnergyScratch {
  double partials[2 * kStaticEnergyBlocks];
  double scal[4];                            // [0] E [1] <psi|psi> [2] Re<psi|H' psi>
  unsigned int counter;
};

static __device__ __align__(256) StaticEnergyScratch g_static_energy;

namespace {

std::mutex g_static_mu;
std::vector<StaticEnergyScratch*> g_static_addr;   // per device ordinal, resolved once

// Device address of g_static_energy on `device`, which must be current.
int static_scratch(int device, StaticEnergyScratch** out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (device >= (int)g_static_addr.size()) g_static_addr.resize(device + 1, nullptr);
  if (!g_static_addr[device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_energy);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(static energy scratch)");
    g_static_addr[device] = (StaticEnergyScratch*)ptr;
  }
  *out = g_static_addr[device];
  return GOCP_OK;
}

template <typename R>
int launch_energy_static(Problem& p, const void* psi, void* hpsi, StaticEnergyScratch* sc, cudaStream_t st) {
  const int grid = apply_grid(p.n_qubits);
  k_apply_h<R><<<grid, kThreads, 0, st>>>(p.dev->t, (const C_t<R>*)psi, (C_t<R>*)hpsi, p.identity,
                                          sc->partials, &sc->counter, sc->scal);
  count_launches(1);
  return cuda_status(cudaGetLastError(), "k_apply_h (static scratch)");
}

}  // namespace

// gocp_energy_static's work, on the problem's device (current): the untiled
// H psi kernel with the reduction scratch in g_static_energy.
int dev_energy_static(Problem& p, const void* psi, void* hpsi, double* out, int mem, cudaStream_t st) {
  const int blocks = apply_grid(p.n_qubits);
  if (blocks > kStaticEnergyBlocks)
    return fail(GOCP_EINVAL, "gocp_energy_static: a state of 2^" + std::to_string(p.n_qubits) +
                                 " amplitudes needs " + std::to_string(blocks) +
                                 " reduction blocks; the static scratch holds 8192 (at most 24 qubits)");
  StaticEnergyScratch* sc = nullptr;
  int rc = static_scratch(p.device, &sc);
  // the block counter must start at zero (the kernel also leaves it at zero)
  if (!rc) rc = cuda_status(cudaMemsetAsync(&sc->counter, 0, sizeof(unsigned int), st), "clear counter");
  if (!rc) rc = p.precision == GOCP_C64 ? launch_energy_static<float>(p, psi, hpsi, sc, st)
                                        : launch_energy_static<double>(p, psi, hpsi, sc, st);
  if (!rc) rc = cuda_status(cudaMemcpyAsync(out, sc->scal, 2 * sizeof(double),
                                            mem == GOCP_MEM_HOST ? cudaMemcpyDeviceToHost
                                                                 : cudaMemcpyDeviceToDevice, st),
                            "copy energy");
  if (!rc && mem == GOCP_MEM_HOST) rc = cuda_status(cudaStreamSynchronize(st), "synchronise");
  return rc;
}

}  // namespace gocp

namespace gocp {

// ------------------------------------------------------------ batched launch

size_t batch_desc_bytes(int n) { return (size_t)n * sizeof(BatchItemDev); }

bool has_tiled_form(const Problem& p) { return p.dev && !p.sector && p.dev->t.n_pieces > 0; }

namespace {

// Blocks one on-chip stage item of this problem takes: 1 (one block's shared
// memory), 2..16 (one cluster), or 0 (the per-step stages).
template <typename R>
int stage_blocks(const Problem& p, int kind) {
  const int states = kind == STAGE_BACKWARD_ALL ? 2 : 1;
  if (smem_chain_fits<R>(*p.dev, states)) return 1;
  const int cb = chain_cluster_blocks<R>(*p.dev, states);
  if (cb <= 0 || smem_chain_optin<R>() != GOCP_OK) return 0;
  const void* k = kind == STAGE_BACKWARD_ALL ? (const void*)k_stage_backward_cluster<R>
                                             : (const void*)k_stage_forward_cluster<R>;
  return cluster_fits(k, cb, ((size_t)states * sizeof(C_t<R>) << p.n_qubits) / cb + kSmemDescBytes) ? cb : 0;
}

}  // namespace

bool stage_onchip(const Problem& p, int kind) {
  if (!p.dev || p.sector) return false;
  return (p.precision == GOCP_C64 ? stage_blocks<float>(p, kind) : stage_blocks<double>(p, kind)) > 0;
}

namespace {

// Blocks of one item: a fixed function of its size and the stage only.
int item_blocks(const Problem& p, int kind) {
  const uint64_t dim = 1ull << p.n_qubits;
  uint64_t want;
  if (kind == STAGE_ENERGY) want = (dim + kTileH - 1) / kTileH;
  else if (kind == STAGE_FORWARD || kind == STAGE_BACKWARD) want = ((dim >> 1) + kThreads - 1) / kThreads;
  else want = (dim + kThreads - 1) / kThreads;
  uint64_t cap = (uint64_t)std::max(p.sm_count, 1) * kItemBlocksPerSm;
  cap = std::min<uint64_t>(cap, kMaxItemBlocks);
  return (int)std::max<uint64_t>(1, std::min(want, cap));
}

template <typename R>
int launch_stage_typed(int kind, const StageItem* items_in, int n, void* host_desc, void* dev_desc,
                       cudaStream_t st, int64_t* launches) {
  // on-chip stages: items ordered by the blocks each takes (one launch per size)
  std::vector<StageItem> sorted;
  const StageItem* items = items_in;
  if (kind == STAGE_FORWARD_ALL || kind == STAGE_BACKWARD_ALL) {
    sorted.assign(items_in, items_in + n);
    std::stable_sort(sorted.begin(), sorted.end(), [&](const StageItem& a, const StageItem& b) {
      return stage_blocks<R>(*a.prob, kind) < stage_blocks<R>(*b.prob, kind);
    });
    items = sorted.data();
  }
  BatchItemDev* hd = (BatchItemDev*)host_desc;
  BatchIndex ix;
  ix.n = n;
  int total = 0;
  for (int i = 0; i < n; ++i) {
    const StageItem& s = items[i];
    const Problem& p = *s.prob;
    BatchItemDev& d = hd[i];
    d.t = p.dev->t;
    d.ops = s.ops;
    d.theta = s.theta;
    d.coefs = s.coefs;
    d.psi = s.psi;
    d.lam = s.lam;
    d.partials = s.partials;
    d.counter = s.counter;
    d.scal = s.scal;
    d.dtheta = s.dtheta;
    d.err = s.err;
    d.identity = p.identity;
    d.ref_index = p.ref_index;
    d.n_ops = s.n_ops;
    d.j = s.j;
    d.nb = item_blocks(p, kind);
    ix.start[i] = total;
    total += d.nb;
  }
  ix.start[n] = total;
  int rc = cuda_status(cudaMemcpyAsync(dev_desc, host_desc, batch_desc_bytes(n), cudaMemcpyHostToDevice, st),
                       "batch descriptors");
  if (rc) return rc;
  const BatchItemDev* dd = (const BatchItemDev*)dev_desc;
  switch (kind) {
    case STAGE_SETUP:
      k_stage_setup<R><<<total, kThreads, 0, st>>>(dd, ix);
      *launches += 1;
      break;
    case STAGE_FORWARD:
      k_stage_forward<R><<<total, kThreads, 0, st>>>(dd, ix);
      *launches += 1;
      break;
    case STAGE_ENERGY:
      // H psi + energy, then lambda = (H psi - E psi)/<psi|psi> once E is known
      k_stage_energy<R><<<total, kThreads, 0, st>>>(dd, ix);
      k_stage_residual<R><<<total, kThreads, 0, st>>>(dd, ix);
      *launches += 2;
      break;
    case STAGE_BACKWARD:
      k_stage_backward<R><<<total, kThreads, 0, st>>>(dd, ix);
      *launches += 1;
      break;
    case STAGE_RESIDUAL:
      k_stage_residual<R><<<total, kThreads, 0, st>>>(dd, ix);
      *launches += 1;
      break;
    case STAGE_FORWARD_ALL:
    case STAGE_BACKWARD_ALL: {
      // items ordered by blocks (1 first, then clusters of 2, 4, 8, 16):
      // one launch per size
      if ((rc = smem_chain_optin<R>())) return rc;
      int i = 0;
      while (i < n) {
        const int nb = stage_blocks<R>(*items[i].prob, kind);
        int e = i;
        while (e < n && stage_blocks<R>(*items[e].prob, kind) == nb) ++e;
        if (nb <= 0) return fail(GOCP_EINVAL, "on-chip stage item does not fit");
        if (nb == 1) {
          if (kind == STAGE_FORWARD_ALL)
            k_stage_forward_all<R><<<e - i, kSmemThreads, kSmemStateBytes + kSmemDescBytes, st>>>(dd + i);
          else
            k_stage_backward_all<R><<<e - i, kSmemThreads, kSmemStateBytes + kSmemDescBytes, st>>>(dd + i);
          if ((rc = cuda_status(cudaGetLastError(), "on-chip stage"))) return rc;
        } else {
          const BatchItemDev* base = dd;
          int first = i;
          void* args[] = {&base, &first};
          if ((rc = launch_cluster(kind == STAGE_FORWARD_ALL ? (const void*)k_stage_forward_cluster<R>
                                                             : (const void*)k_stage_backward_cluster<R>,
                                   nb, kSmemStateBytes + kSmemDescBytes, args, st, e - i)))
            return rc;
        }
        *launches += 1;
        i = e;
      }
      break;
    }
    default:
      return fail(GOCP_EINVAL, "unknown stage kind");
  }
  return cuda_status(cudaGetLastError(), "batched stage");
}

}  // namespace

int launch_stage(int kind, const StageItem* items, int n, int precision, void* host_desc,
                 void* dev_desc, void* stream, int64_t* launches) {
  if (n <= 0) return GOCP_OK;
  if (n > kMaxBatchItems) return fail(GOCP_EINVAL, "too many items in one batch");
  int64_t before = *launches;
  int rc = precision == GOCP_C64
               ? launch_stage_typed<float>(kind, items, n, host_desc, dev_desc, (cudaStream_t)stream, launches)
               : launch_stage_typed<double>(kind, items, n, host_desc, dev_desc, (cudaStream_t)stream, launches);
  count_launches(*launches - before);
  return rc;
}

}  // namespace gocp
