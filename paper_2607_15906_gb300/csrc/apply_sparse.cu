// H psi (Eq. 3) with the energy epilogue (Eq. 1) for states with few
// nonzero amplitudes, by scattering from the nonzero source amplitudes.
//
// The staged kernel (apply_tiled.cu) gives every thread an output octet and
// walks the groups of a piece, skipping a group only where the whole source
// octet is zero; in a state confined to a particle-number sector (1.5 % of
// the amplitudes nonzero at 24 qubits, in 8.9 % of the octets) most lanes of
// a warp idle while a few work.  This kernel turns the loop around:
//
//  * a listing pass writes the nonzero amplitudes (index, value) in index
//    order, and the first entry of every tile;
//  * a block (one per SM) owns an output tile t of 2^LB amplitudes and
//    accumulates it in shared memory.  Its work units are (piece, chunk): 32
//    consecutive nonzero amplitudes of the piece's source tile
//    u = t ^ (x >> LB), one per lane, against the piece's groups, which the
//    warp walks together from its own shared-memory copy of the piece's
//    blob.  Units are numbered piece by piece from a per-tile scan of chunk
//    counts and claimed a few at a time.  For a group with mask x the lane's
//    amplitude psi(k') goes to output k = k' ^ x with weight D(k): a LUT
//    group reads its entry at code(k) (the code is linear in k over GF(2)),
//    a term-list group sums its terms' signs at k (times the factor 0 or 2
//    of a paired group).  A nonzero product is added to the accumulator with
//    a shared-memory atomic; a zero weight adds nothing and is left out;
//  * after the last unit, lanes over the nonzero amplitudes of the own tile
//    add the diagonal group and the identity and take the energy partials;
//    then the whole tile (zeros included) is streamed to H psi.
//
// Every lane does the same work for every group, whatever the sparsity
// pattern, and a group's descriptor and LUT are read at one address per
// warp.  The order in which products reach an accumulator element is not
// fixed, so the result may differ from run to run in the last bits of a sum
// (and from the staged kernel's order); every term is the same.
//
// The kernel is launched with the staged one; each returns at once unless
// the count of nonzero amplitudes selects it, so the choice needs no host
// round trip.
#include <algorithm>
#include <mutex>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace gocp {

namespace {

constexpr int kAmpBlock = 256;   // listing passes: one amplitude word (4 octets) per thread
constexpr uint32_t kUnitBatch = 4;   // scatter work units per claim

// One block per SM: 1024 threads for complex64 (64 registers), 512 for
// complex128 (128 registers).
template <typename R>
__host__ __device__ constexpr int sp_threads() { return sizeof(R) == 4 ? 1024 : 512; }

template <typename R>
__device__ __forceinline__ void load_octet(const C_t<R>* __restrict__ psi, uint32_t octet, C_t<R> (&v)[kAmpsH]) {
  if (sizeof(R) == 4) {
    const float4* p = reinterpret_cast<const float4*>(psi) + (size_t)octet * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 f = __ldg(p + q);
      v[2 * q] = cmake<R>((R)f.x, (R)f.y);
      v[2 * q + 1] = cmake<R>((R)f.z, (R)f.w);
    }
  } else {
    const double2* p = reinterpret_cast<const double2*>(psi) + (size_t)octet * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double2 f = __ldg(p + q);
      v[q] = cmake<R>((R)f.x, (R)f.y);
    }
  }
}

template <typename R>
__device__ __forceinline__ uint32_t nonzero_members(const C_t<R> (&v)[kAmpsH]) {
  uint32_t nz = 0;
#pragma unroll
  for (int m = 0; m < kAmpsH; ++m) nz |= (uint32_t)(v[m].x != R(0) || v[m].y != R(0)) << m;
  return nz;
}

// Members of octet o nonzero in psi or (when set) psi2.
template <typename R>
__device__ __forceinline__ uint32_t octet_nonzero2(const C_t<R>* __restrict__ psi, const C_t<R>* __restrict__ psi2,
                                                   uint32_t o) {
  C_t<R> v[kAmpsH];
  load_octet<R>(psi, o, v);
  uint32_t nz = nonzero_members<R>(v);
  if (psi2) {
    load_octet<R>(psi2, o, v);
    nz |= nonzero_members<R>(v);
  }
  return nz;
}

// Amplitude word w: bit 8j + i = member i of octet 4w + j nonzero in psi or
// (when set) psi2, read only from the octets the octet mask marks live.
template <typename R>
__device__ __forceinline__ uint32_t amp_word(const C_t<R>* __restrict__ psi, const C_t<R>* __restrict__ psi2,
                                             const uint32_t* __restrict__ mask, uint32_t w) {
  const uint32_t mb = (mask[w >> 3] >> ((w & 7u) * 4u)) & 0xFu;
  uint32_t word = 0;
#pragma unroll
  for (uint32_t j = 0; j < 4; ++j)
    if ((mb >> j) & 1u) word |= octet_nonzero2<R>(psi, psi2, 4u * w + j) << (8u * j);
  return word;
}

// counts[b] = the amplitudes nonzero in psi or psi2 in amplitude words
// kAmpBlock b .. kAmpBlock (b + 1) - 1 (one thread per word of 32).
template <typename R>
__global__ void __launch_bounds__(kAmpBlock)
k_amp_count(const C_t<R>* __restrict__ psi, const C_t<R>* __restrict__ psi2, const uint32_t* __restrict__ mask,
            uint32_t words, uint32_t* counts) {
  __shared__ uint32_t red[kAmpBlock / 32];
  const uint32_t w = blockIdx.x * kAmpBlock + threadIdx.x;
  uint32_t c = w < words ? __popc(amp_word<R>(psi, psi2, mask, w)) : 0u;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int q = 0; q < kAmpBlock / 32; ++q) t += red[q];
    counts[blockIdx.x] = t;
  }
}

// counts[0..nb) -> exclusive prefix sums in place; *total = the sum (when
// set; and, when ring is set, the chain-list ring's base(slot) = the sum,
// count(slot) = count(first) = 0).  One block of 1024 threads.
__global__ void __launch_bounds__(1024)
k_amp_scan(uint32_t* counts, uint32_t nb, uint32_t* total, uint32_t* ring, int slot, int first) {
  __shared__ uint32_t s[1024];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  for (uint32_t base = 0; base < nb; base += 1024u) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < nb ? counts[i] : 0u;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {   // inclusive scan
      const uint32_t u = (int)threadIdx.x >= d ? s[threadIdx.x - d] : 0u;
      __syncthreads();
      s[threadIdx.x] += u;
      __syncthreads();
    }
    if (i < nb) counts[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (total) *total = carry;
    if (ring) {
      ring[kRingBase(slot)] = carry;
      ring[kRingAdd(slot)] = 0u;
      ring[kRingAdd(first)] = 0u;
    }
  }
}

// Writes the index (and, when aval is set, the psi value) of every amplitude
// nonzero in psi or psi2, in index order, at the offsets of k_amp_scan;
// entries at or beyond cap are not stored.  With amask set, also writes
// amask[w] = amplitude word w (one bit per amplitude, zeros included).
template <typename R>
__global__ void __launch_bounds__(kAmpBlock)
k_amp_list(const C_t<R>* __restrict__ psi, const C_t<R>* __restrict__ psi2, const uint32_t* __restrict__ mask,
           uint32_t words, const uint32_t* __restrict__ offs, uint32_t* aidx, C_t<R>* aval, uint32_t* amask,
           uint32_t cap) {
  __shared__ uint32_t red[kAmpBlock / 32];
  const uint32_t w = blockIdx.x * kAmpBlock + threadIdx.x;
  const uint32_t word = w < words ? amp_word<R>(psi, psi2, mask, w) : 0u;
  const uint32_t c = __popc(word);
  // exclusive scan over the block: lanes by shuffles, warps through red
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = c;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) red[warp] = incl;
  __syncthreads();
  uint32_t before = 0;
  for (int q = 0; q < warp; ++q) before += red[q];
  uint32_t at = offs[blockIdx.x] + before + incl - c;
  for (uint32_t m = word; m; m &= m - 1u, ++at) {
    if (at >= cap) break;
    const uint32_t k = 32u * w + (uint32_t)(__ffs(m) - 1);
    aidx[at] = k;
    if (aval) aval[at] = psi[k];
  }
  if (amask && w < words) amask[w] = word;
}

// off[u] = first stored entry with index >> shift >= u, u = 0 .. ntiles
// (off[ntiles] = the number of stored entries).
__global__ void __launch_bounds__(256)
k_tile_offsets(const uint32_t* __restrict__ idx, const uint32_t* __restrict__ len, uint32_t cap, uint32_t ntiles,
               int shift, uint32_t* off) {
  const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u > ntiles) return;
  uint32_t lo = 0, hi = min(*len, cap);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((idx[mid] >> shift) < u) lo = mid + 1;
    else hi = mid;
  }
  off[u] = lo;
}

// The tile's accumulator holds component j (2i: real part, 2i + 1:
// imaginary part of member i) of octet o at j kOct + (o ^ 4i): a warp's
// atomics on one component spread over the banks by octet, two members of
// one octet fall on different banks, and the epilogue's reads of one
// component stay a permutation of 32 consecutive words.
template <uint32_t kOct>
__device__ __forceinline__ uint32_t acc_at(uint32_t k) {
  const uint32_t i = k & 7u, o = (k >> 3) & (kOct - 1u);
  return (2u * i) * kOct + (o ^ (i << 2));
}

template <typename R, uint32_t kOct>
__device__ __forceinline__ void acc_add(R* acc, uint32_t k, R re, R im) {
  const uint32_t at = acc_at<kOct>(k);
  atomicAdd(acc + at, re);
  atomicAdd(acc + at + kOct, im);
}

// One LUT group against the lane's nonzero amplitude psi(ks) = v.  The
// entry's magnitude depends on phi(k) alone (lut16[phi | 8] = -lut16[phi]),
// so the sign parity is taken only for a nonzero entry.
template <typename R, uint32_t kOct>
__device__ __forceinline__ void sp_lut(const HLut<R>& L, uint32_t ks, C_t<R> v, bool valid, R* acc) {
  const uint4 h0 = *reinterpret_cast<const uint4*>(&L.x);     // x, z0, v0, v1
  const uint32_t v2 = L.v2;
  const uint32_t k = ks ^ h0.x;
  const uint32_t phi = (uint32_t)(__popc(k & h0.z) & 1) | ((uint32_t)(__popc(k & h0.w) & 1) << 1) |
                       ((uint32_t)(__popc(k & v2) & 1) << 2);
  const R d0 = L.lut16[phi];
  if (valid && d0 != R(0)) {
    const R d = (__popc(k & h0.y) & 1) ? -d0 : d0;
    acc_add<R, kOct>(acc, k, d * v.x, d * v.y);
  }
}

// One term-list group: D(k) = sum_t w_t (-1)^popc(k & z_t), real terms
// [tb, tm), imaginary [tm, te); a paired group keeps one term of each pair
// and D = (1 + sigma (-1)^popc(k & delta)) E(k), the factor 0 or 2.  Called
// by every lane of the warp (the group is warp-uniform).
template <typename R, uint32_t kOct>
__device__ __forceinline__ void sp_terms(const TiledGroup& G, const uint32_t* __restrict__ zs,
                                         const R* __restrict__ ws, uint32_t ks, C_t<R> v, bool valid, R* acc) {
  const uint32_t k = ks ^ G.x;
  R f = R(1);
  if (G.delta) {
    const uint32_t p = __popc(k & G.delta) & 1u;
    f = (G.neg ? p : p ^ 1u) ? R(2) : R(0);
  }
  const bool on = valid && f != R(0);
  if (!__any_sync(0xffffffffu, on)) return;
  R dr = R(0), di = R(0);
  for (uint32_t t = G.tb; t < G.tm; ++t) dr += (__popc(k & zs[t]) & 1) ? -ws[t] : ws[t];
  for (uint32_t t = G.tm; t < G.te; ++t) di += (__popc(k & zs[t]) & 1) ? -ws[t] : ws[t];
  dr *= f;
  di *= f;
  if (on && (dr != R(0) || di != R(0))) acc_add<R, kOct>(acc, k, dr * v.x - di * v.y, dr * v.y + di * v.x);
}

template <typename R>
__global__ void __launch_bounds__(sp_threads<R>(), 1) k_apply_h_sparse(const SparseArgs<R> a) {
  constexpr int LB = TiledBits<R>::LB;
  constexpr int NT = sp_threads<R>();
  constexpr uint32_t kOct = 1u << (LB - 3);   // octets per tile
  if (*a.alen > a.max_amps) return;           // the staged kernel takes this state
  // dynamic shared memory: the tile's accumulator (16 components x kOct
  // octets), then one piece blob per warp
  extern __shared__ __align__(16) uint8_t sp_raw[];
  R* acc = reinterpret_cast<R*>(sp_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t* wblob = sp_raw + kOct * 16u * sizeof(R) + (size_t)warp * kTiledBlobBytes;
  __shared__ uint32_t s_tile, s_unext;
  __shared__ uint32_t s_pre[kSpMaxPieces + 1];   // first unit of each piece; s_pre[P] = units
  __shared__ uint32_t s_wsum[32];
  __shared__ double tot[2];
  const uint32_t ntiles = 1u << (a.n - LB);
  const uint32_t P = (uint32_t)a.n_pieces;
  for (uint32_t j = threadIdx.x; j < kOct * 16u; j += NT) acc[j] = R(0);
  const R idr = (R)a.identity;
  // this thread's |psi|^2 and <psi|H - identity|psi> partials (in shared
  // memory: touched once per tile)
  __shared__ double2 s_v[NT];
  s_v[threadIdx.x] = make_double2(0.0, 0.0);
  for (;;) {
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(a.tile_counter, 1u);
      s_unext = 0u;
    }
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= ntiles) break;
    // Work units are (piece p, chunk c): the nonzero amplitudes 32c .. 32c + 31
    // of p's source tile u = t ^ (x >> LB) against p's groups, numbered piece
    // by piece (s_pre: a block scan of the chunk counts).
    {
      const uint32_t per = (P + NT - 1) / NT, p0 = threadIdx.x * per, p1 = min(P, p0 + per);
      uint32_t mine = 0;
      for (uint32_t p = p0; p < p1; ++p) {
        const TiledPiece pc = a.piece[p];
        const uint32_t u = t ^ pc.xhi;
        const uint32_t nch = pc.bytes ? (a.toff[u + 1] - a.toff[u] + 31u) >> 5 : 0u;
        s_pre[p] = nch;
        mine += nch;
      }
      uint32_t incl = mine;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t q = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += q;
      }
      if (lane == 31) s_wsum[warp] = incl;
      __syncthreads();
      if (warp == 0) {
        uint32_t w = lane < NT / 32 ? s_wsum[lane] : 0u, wi = w;
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t q = __shfl_up_sync(0xffffffffu, wi, o);
          if (lane >= o) wi += q;
        }
        if (lane < NT / 32) s_wsum[lane] = wi - w;   // exclusive
        if (lane == NT / 32 - 1) s_pre[P] = wi;
      }
      __syncthreads();
      uint32_t run = s_wsum[warp] + incl - mine;
      for (uint32_t p = p0; p < p1; ++p) {
        const uint32_t nch = s_pre[p];
        s_pre[p] = run;
        run += nch;
      }
    }
    __syncthreads();
    const uint32_t n_units = s_pre[P];
    uint32_t cur = 0xFFFFFFFFu;   // piece whose blob this warp holds
    for (;;) {
      // kUnitBatch consecutive units per claim: mostly chunks of one piece,
      // whose blob is then copied once
      uint32_t j0 = 0;
      if (lane == 0) j0 = atomicAdd(&s_unext, kUnitBatch);
      j0 = __shfl_sync(0xffffffffu, j0, 0);
      if (j0 >= n_units) break;
      const uint32_t j1 = min(n_units, j0 + kUnitBatch);
      // p = the last piece with s_pre[p] <= j0 (pieces without units share
      // their successor's start and are passed over), then advanced along
      // the batch
      uint32_t p;
      {
        uint32_t lo = 0, hi = P - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (s_pre[mid] <= j0) lo = mid;
          else hi = mid - 1;
        }
        p = lo;
      }
      for (uint32_t j = j0; j < j1; ++j) {
      while (p + 1 < P && s_pre[p + 1] <= j) ++p;
      const uint32_t c = j - s_pre[p];
      const TiledPiece pc = a.piece[p];
      if (p != cur) {
        // the piece's blob into this warp's buffer, 16 bytes per lane
        __syncwarp();
        const uint4* src = reinterpret_cast<const uint4*>(a.blob + pc.off);
        uint4* dst = reinterpret_cast<uint4*>(wblob);
        for (uint32_t q = (uint32_t)lane; q < pc.bytes / 16u; q += 32u) dst[q] = __ldg(src + q);
        __syncwarp();
        cur = p;
      }
      const uint32_t u = t ^ pc.xhi;
      const uint32_t a0 = a.toff[u], a1 = a.toff[u + 1];
      const TiledHead* hd = reinterpret_cast<const TiledHead*>(wblob);
      const HLut<R>* ls = reinterpret_cast<const HLut<R>*>(wblob + sizeof(TiledHead));
      const TiledGroup* gs =
          reinterpret_cast<const TiledGroup*>(wblob + sizeof(TiledHead) + hd->n_lut * sizeof(HLut<R>));
      const uint32_t* zs = reinterpret_cast<const uint32_t*>(wblob + hd->z_off);
      const R* ws = reinterpret_cast<const R*>(wblob + hd->w_off);
      const uint32_t li = a0 + 32u * c + (uint32_t)lane;
      const bool valid = li < a1;
      const uint32_t ks = a.aidx[valid ? li : a0];
      const C_t<R> v = a.aval[valid ? li : a0];
      const int nl = (int)hd->n_lut;
      for (int g = 0; g < nl; ++g) sp_lut<R, kOct>(ls[g], ks, v, valid, acc);
      // the term-list groups fill the blob from the LUT groups to z_off
      const int nt = (int)((hd->z_off - sizeof(TiledHead) - nl * sizeof(HLut<R>)) / sizeof(TiledGroup));
      for (int g = 0; g < nt; ++g) sp_terms<R, kOct>(gs[g], zs, ws, ks, v, valid, acc);
      }
    }
    __syncthreads();
    // epilogue, first the nonzero amplitudes of the own tile (one lane
    // each): the diagonal group and the identity, which act on psi(k) alone,
    // and the energy partials (zero amplitudes add to neither); each k is
    // one lane's, so its accumulator entry is updated without atomics
    {
      const uint32_t e0 = a.toff[t], e1 = a.toff[t + 1];
      double2 w = s_v[threadIdx.x];
      for (uint32_t e = e0 + threadIdx.x; e < e1; e += NT) {
        const uint32_t k = a.aidx[e];
        const C_t<R> q = a.aval[e];
        R dr = R(0), dc = R(0), di = R(0);
        for (int m = 0; m < a.nd_mid; ++m) {
          const R y = ((__popc(k & a.dz[m]) & 1) ? -a.dw[m] : a.dw[m]) - dc;
          if (sizeof(R) == 4) {   // compensated in FP32
            const R s2 = dr + y;
            dc = (s2 - dr) - y;
            dr = s2;
          } else {
            dr += y;
          }
        }
        for (int m = a.nd_mid; m < a.nd; ++m) di += (__popc(k & a.dz[m]) & 1) ? -a.dw[m] : a.dw[m];
        R* e2 = acc + acc_at<kOct>(k);
        const C_t<R> off = cmake<R>(e2[0], e2[kOct]);
        const double pp = (double)q.x * q.x + (double)q.y * q.y;
        w.x += pp;
        w.y += (double)q.x * off.x + (double)q.y * off.y + ((double)dr - (double)dc) * pp;
        const R d0 = dr - dc + idr;
        e2[0] = off.x + d0 * q.x - di * q.y;
        e2[kOct] = off.y + d0 * q.y + di * q.x;
      }
      s_v[threadIdx.x] = w;
    }
    __syncthreads();
    // then the whole tile out (zeros included) and the accumulator cleared
    for (uint32_t o = threadIdx.x; o < kOct; o += NT) {
      const uint32_t k0 = ((t << (LB - 3)) | o) << 3;
      C_t<R> res[kAmpsH];
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) {
        R* e = acc + acc_at<kOct>(k0 | (uint32_t)i);
        res[i] = cmake<R>(e[0], e[kOct]);
        e[0] = R(0);
        e[kOct] = R(0);
      }
      C_t<R>* dst = a.out + k0;
      if (sizeof(R) == 4) {
        float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
        for (int q = 0; q < kAmpsH / 2; ++q)
          __stcs(d4 + q, make_float4((float)res[2 * q].x, (float)res[2 * q].y, (float)res[2 * q + 1].x,
                                     (float)res[2 * q + 1].y));
      } else {
        double2* d2 = reinterpret_cast<double2*>(dst);
#pragma unroll
        for (int q = 0; q < kAmpsH; ++q) __stcs(d2 + q, make_double2((double)res[q].x, (double)res[q].y));
      }
    }
    __syncthreads();
  }
  const double v[2] = {s_v[threadIdx.x].x, s_v[threadIdx.x].y};
  if (a.partials && block_grid_sum<2, NT>(v, a.partials, a.counter, gridDim.x, blockIdx.x, a.scal + 1, tot)) {
    if (threadIdx.x == 0) a.scal[0] = a.identity + tot[1] / tot[0];
  }
}

template <typename R>
constexpr uint32_t sparse_smem() {
  return (1u << (TiledBits<R>::LB - 3)) * 16u * (uint32_t)sizeof(R) + (sp_threads<R>() / 32) * kTiledBlobBytes;
}

}  // namespace

template <typename R>
int sparse_apply_h(SparseArgs<R> a, const LiveOctets& lv, int sm_count, cudaStream_t st) {
  constexpr int LB = TiledBits<R>::LB;
  if (a.n < LB || !lv.toff || !lv.aidx || !lv.aval || !lv.alen || !lv.acounts || a.max_amps > lv.acap)
    return fail(GOCP_EINVAL, "scatter H psi needs the amplitude list");
  a.aidx = lv.aidx;
  a.aval = reinterpret_cast<const C_t<R>*>(lv.aval);
  a.alen = lv.alen;
  a.toff = lv.toff;
  static std::mutex mu;
  static std::vector<bool> done;
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  {
    std::lock_guard<std::mutex> lk(mu);
    if (device >= (int)done.size()) done.resize(device + 1, false);
    if (!done[device]) {
      e = cudaFuncSetAttribute(k_apply_h_sparse<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sparse_smem<R>());
      if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_apply_h_sparse)");
      done[device] = true;
    }
  }
  int rc = amp_list(sizeof(R) == 4 ? GOCP_C64 : GOCP_C128, a.psi, a.mask, a.n, lv, st);
  if (rc) return rc;
  const uint32_t ntiles = 1u << (a.n - LB);
  k_tile_offsets<<<(ntiles + 256u) / 256u, 256, 0, st>>>(lv.aidx, lv.alen, lv.acap, ntiles, LB, lv.toff);
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)std::max(sm_count, 1));
  k_apply_h_sparse<R><<<grid, sp_threads<R>(), sparse_smem<R>(), st>>>(a);
  count_launches(2);
  return cuda_status(cudaGetLastError(), "k_apply_h_sparse");
}

int amp_list(int precision, const void* psi, const uint32_t* mask, int n, const LiveOctets& lv, cudaStream_t st) {
  if (n < 8 || !mask || !lv.aidx || !lv.aval || !lv.alen || !lv.acounts)
    return fail(GOCP_EINVAL, "amplitude list needs n >= 8 and its buffers");
  const uint32_t words = 1u << (n - 5);   // amplitude words
  const uint32_t nb = (words + kAmpBlock - 1u) / kAmpBlock;
  if (precision == GOCP_C64) {
    const float2* p = reinterpret_cast<const float2*>(psi);
    k_amp_count<float><<<nb, kAmpBlock, 0, st>>>(p, nullptr, mask, words, lv.acounts);
    k_amp_scan<<<1, 1024, 0, st>>>(lv.acounts, nb, lv.alen, nullptr, 0, 0);
    k_amp_list<float><<<nb, kAmpBlock, 0, st>>>(p, nullptr, mask, words, lv.acounts, lv.aidx,
                                                reinterpret_cast<float2*>(lv.aval), nullptr, lv.acap);
  } else {
    const double2* p = reinterpret_cast<const double2*>(psi);
    k_amp_count<double><<<nb, kAmpBlock, 0, st>>>(p, nullptr, mask, words, lv.acounts);
    k_amp_scan<<<1, 1024, 0, st>>>(lv.acounts, nb, lv.alen, nullptr, 0, 0);
    k_amp_list<double><<<nb, kAmpBlock, 0, st>>>(p, nullptr, mask, words, lv.acounts, lv.aidx,
                                                 reinterpret_cast<double2*>(lv.aval), nullptr, lv.acap);
  }
  count_launches(3);
  return cuda_status(cudaGetLastError(), "k_amp_list");
}

int chain_list(int precision, const void* psi, const void* lam, const uint32_t* mask, int n, const ChainList& cl,
               uint32_t* counts, int slot, int first, cudaStream_t st) {
  if (n < 8 || !mask || !cl.list || !cl.amask || !cl.cnt || !counts)
    return fail(GOCP_EINVAL, "chain list needs n >= 8 and its buffers");
  const uint32_t words = 1u << (n - 5);   // amplitude words
  const uint32_t nb = (words + kAmpBlock - 1u) / kAmpBlock;
  if (precision == GOCP_C64) {
    const float2* p = reinterpret_cast<const float2*>(psi);
    const float2* q = reinterpret_cast<const float2*>(lam);
    k_amp_count<float><<<nb, kAmpBlock, 0, st>>>(p, q, mask, words, counts);
    k_amp_scan<<<1, 1024, 0, st>>>(counts, nb, nullptr, cl.cnt, slot, first);
    k_amp_list<float><<<nb, kAmpBlock, 0, st>>>(p, q, mask, words, counts, cl.list, nullptr, cl.amask, cl.cap);
  } else {
    const double2* p = reinterpret_cast<const double2*>(psi);
    const double2* q = reinterpret_cast<const double2*>(lam);
    k_amp_count<double><<<nb, kAmpBlock, 0, st>>>(p, q, mask, words, counts);
    k_amp_scan<<<1, 1024, 0, st>>>(counts, nb, nullptr, cl.cnt, slot, first);
    k_amp_list<double><<<nb, kAmpBlock, 0, st>>>(p, q, mask, words, counts, cl.list, nullptr, cl.amask, cl.cap);
  }
  count_launches(3);
  return cuda_status(cudaGetLastError(), "chain list");
}

template int sparse_apply_h<float>(SparseArgs<float>, const LiveOctets&, int, cudaStream_t);
template int sparse_apply_h<double>(SparseArgs<double>, const LiveOctets&, int, cudaStream_t);

}  // namespace gocp
