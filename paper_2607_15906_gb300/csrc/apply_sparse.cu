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
//    accumulates it in shared memory.  Its work units are (piece, chunk):
//    32 sp_amps consecutive nonzero amplitudes of the piece's source tile
//    u = t ^ (x >> LB), sp_amps per lane, against the piece's groups, which
//    the warp walks together.  Units are numbered piece by piece from a
//    per-tile scan of chunk counts and claimed a few at a time.  For a group with mask x the lane's
//    amplitude psi(k') goes to output k = k' ^ x with weight D(k): a LUT
//    group reads its entry at code(k) (the code is linear in k over GF(2)),
//    a term-list group sums its terms' signs at k (times the factor 0 or 2
//    of a paired group).  A nonzero product is added to the accumulator, in
//    64-bit fixed point, with shared-memory integer atomics; a zero weight
//    adds nothing and is left out.  For complex128 a LUT group's nonzero
//    (amplitude, weight) items are first packed into a per-warp buffer and
//    multiplied and added 32 at a time, so that the FP64 products and
//    conversions run with every lane busy (about two thirds of the items of
//    a sector-confined state have a zero weight);
//  * after the last unit, lanes over the nonzero amplitudes of the own tile
//    add the diagonal group and the identity and take the energy partials;
//    then the whole tile (zeros included) is streamed to H psi.
//
// Every lane does the same work for every group, whatever the sparsity
// pattern, and a group's descriptor and LUT are read at one address per
// warp (from global memory through L1).  The order in which products reach
// an accumulator element is not fixed, but integer addition does not depend
// on it: H psi, E and everything computed from them are reproducible bit
// for bit from run to run.
//
// The kernel is launched with the staged one; each returns at once unless
// the count of nonzero amplitudes selects it, so the choice needs no host
// round trip.
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace gocp {

namespace {

constexpr int kAmpBlock = 256;   // listing passes: one amplitude word (4 octets) per thread
constexpr uint32_t kUnitBatch = 4;   // scatter work units per claim

// Nonzero source amplitudes per lane per work unit: complex64 two, with
// FP32 products added at once; complex128 one, with integer products of the
// fixed-point weights and amplitudes, its LUT-group items compacted per warp
// (see sp_lut_q).
template <typename R>
__host__ __device__ constexpr int sp_amps() { return sizeof(R) == 4 ? 2 : 1; }

// One block of 1024 threads (64 registers) per SM in both precisions
// (complex128 measured 6.3 ms per 24-qubit call at 1024 threads, 6.6 at
// 768, 7.8 at 512).
template <typename R>
__host__ __device__ constexpr int sp_threads() { return 1024; }


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
// count(slot) = count(first) = 0); *amax = 0 when set.  One block of 1024
// threads.  The sum reaches 2^32 only for a 32-qubit state with every
// amplitude nonzero; it is stored saturated at 2^32 - 1 (above every list
// capacity, so the list is not used), while every prefix, at most the sum
// less the last block's count, fits 32 bits.
__global__ void __launch_bounds__(1024)
k_amp_scan(uint32_t* counts, uint32_t nb, uint32_t* total, uint32_t* ring, int slot, int first,
           unsigned long long* amax) {
  __shared__ uint32_t s[1024];
  __shared__ unsigned long long carry;
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
    if (i < nb) counts[i] = (uint32_t)(carry + s[threadIdx.x] - v);
    __syncthreads();
    if (threadIdx.x == 0) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const uint32_t sum = carry > 0xffffffffull ? 0xffffffffu : (uint32_t)carry;
    if (total) *total = sum;
    if (amax) *amax = 0ull;
    if (ring) {
      ring[kRingBase(slot)] = sum;
      ring[kRingAdd(slot)] = 0u;
      ring[kRingAdd(first)] = 0u;
    }
  }
}

// Writes the index (and, when aval is set, the psi value) of every amplitude
// nonzero in psi or psi2, in index order, at the offsets of k_amp_scan;
// entries at or beyond cap are not stored.  With amask set, also writes
// amask[w] = amplitude word w (one bit per amplitude, zeros included).  With
// amax set, raises *amax to the largest |Re| or |Im| of the listed psi values
// (the bits of a non-negative double, which order as unsigned integers).
template <typename R>
__global__ void __launch_bounds__(kAmpBlock)
k_amp_list(const C_t<R>* __restrict__ psi, const C_t<R>* __restrict__ psi2, const uint32_t* __restrict__ mask,
           uint32_t words, const uint32_t* __restrict__ offs, uint32_t* aidx, C_t<R>* aval, uint32_t* amask,
           uint32_t cap, unsigned long long* amax) {
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
  R big = R(0);
  for (uint32_t m = word; m; m &= m - 1u, ++at) {
    if (at >= cap) break;
    const uint32_t k = 32u * w + (uint32_t)(__ffs(m) - 1);
    aidx[at] = k;
    if (aval) {
      const C_t<R> v = psi[k];
      aval[at] = v;
      big = fmax(big, fmax(fabs(v.x), fabs(v.y)));
    }
  }
  if (amask && w < words) amask[w] = word;
  if (amax) {
    for (int o = 16; o > 0; o >>= 1) big = fmax(big, __shfl_xor_sync(0xffffffffu, big, o));
    if (lane == 0 && big > R(0)) atomicMax(amax, (unsigned long long)__double_as_longlong((double)big));
  }
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

// Fixed-point accumulation.  A product p is added as the integer
// round(p 2^F) (the amplitudes are scaled by 2^F once, see below), so the
// sum is exact integer arithmetic: the same in any order of the atomics,
// and the result is bit-for-bit reproducible.  F is chosen per call so that
// the sum of the magnitudes of all contributions to one output component --
// at most hbound x 2 max(|Re psi|, |Im psi|) -- stays below 2^62: no partial
// sum can overflow.  For complex64, F also keeps every off-diagonal product
// below 2^30, so that it converts with a 32-bit instruction; its rounding,
// at most 2^-(F+1), is then about 1e-9 of the largest possible product, and
// an entry of H psi collects it from at most a few thousand products.  For
// complex128 the rounding is at most 2^-(F+1) with F near 62 - log2 of the
// bound, far below the FP64 rounding of the products.

// Adds v to the 64-bit accumulator word p as two 32-bit atomics: the low
// word's, and the high word's plus the carry out of the low word, taken from
// the old value that atomic returns.  The pair is exact modulo 2^64 in any
// order of the atomics (measured faster than one 64-bit atomic).  complex128
// adds its products this way; complex64 uses the split form (fx_add_split).
__device__ __forceinline__ void fx_add(unsigned long long* p, long long v) {
  uint32_t* w = reinterpret_cast<uint32_t*>(p);
  const uint32_t lo = (uint32_t)(unsigned long long)v, hi = (uint32_t)((unsigned long long)v >> 32);
  const uint32_t old = atomicAdd(w, lo);
  atomicAdd(w + 1, hi + (uint32_t)(old + lo < old));
}

// A scaled product as an integer.  complex64: every off-diagonal product is
// below 2^30 by the choice of F, so a 32-bit conversion suffices (the 64-bit
// conversions run on the FP64 pipe, narrow on this part); complex128: FP64
// products, a 64-bit conversion.
template <typename R>
__device__ __forceinline__ long long fx_prod(R v) {
  return sizeof(R) == 4 ? (long long)__float2int_rn((float)v) : __double2ll_rn((double)v);
}

// A scaled value up to 2^62 (the diagonal's products, once per amplitude).
template <typename R>
__device__ __forceinline__ long long fx_wide(R v) {
  return sizeof(R) == 4 ? __float2ll_rn((float)v) : __double2ll_rn((double)v);
}

// An accumulator value back in R (zeros, most of a sector state's tile,
// skip the conversion).
template <typename R>
__device__ __forceinline__ R fx_val(unsigned long long a) {
  if (a == 0ull) return R(0);
  return sizeof(R) == 4 ? (R)__ll2float_rn((long long)a) : (R)__ll2double_rn((long long)a);
}

// Split form of the accumulator word (complex64, products below 2^30): its
// low 32-bit half sums the low 16 bits of each product (0 .. 65535) and its
// high half the product shifted right by 16 (arithmetic, |.| <= 2^14), two
// independent atomics with no carry between them.  With fewer than 65536
// products per word (one per off-diagonal group) neither half can wrap:
// low < 2^16 * 65536 = 2^32, |high| < 2^30.  The word's value is
// high * 2^16 + low, formed exactly by split_to_wide once every product has
// been added.
__device__ __forceinline__ void fx_add_split(unsigned long long* p, int v) {
  uint32_t* w = reinterpret_cast<uint32_t*>(p);
  atomicAdd(w, (uint32_t)v & 0xFFFFu);
  atomicAdd(w + 1, (uint32_t)(v >> 16));
}

__device__ __forceinline__ unsigned long long split_to_wide(unsigned long long w) {
  const long long high = (long long)(int)(uint32_t)(w >> 32);
  return (unsigned long long)(high * 65536ll + (long long)(w & 0xffffffffull));
}

template <uint32_t kOct, bool SPLIT = false>
__device__ __forceinline__ void acc_add(unsigned long long* acc, uint32_t k, long long re, long long im) {
  const uint32_t at = acc_at<kOct>(k);
  if constexpr (SPLIT) {
    fx_add_split(acc + at, (int)re);
    fx_add_split(acc + at + kOct, (int)im);
  } else {
    fx_add(acc + at, re);
    fx_add(acc + at + kOct, im);
  }
}

// One LUT group (descriptor in global memory, read through L1 at one
// address per warp) against the lane's nonzero amplitudes psi(ks[s]), whose
// values vs[s] are pre-scaled by 2^F.  The entry's magnitude depends on
// phi(k) alone (lut16[phi | 8] = -lut16[phi]), so the sign parity is taken
// only for a nonzero entry.
template <typename R, uint32_t kOct, int A, bool SPLIT>
__device__ __forceinline__ void sp_lut(const HLut<R>* __restrict__ L, const uint4 h0, const uint32_t v2,
                                       const uint32_t (&ks)[A], const C_t<R> (&vs)[A], const bool (&valid)[A],
                                       unsigned long long* acc) {
#pragma unroll
  for (int s = 0; s < A; ++s) {
    const uint32_t k = ks[s] ^ h0.x;
    const uint32_t phi = (uint32_t)(__popc(k & h0.z) & 1) | ((uint32_t)(__popc(k & h0.w) & 1) << 1) |
                         ((uint32_t)(__popc(k & v2) & 1) << 2);
    const R d0 = __ldg(L->lut16 + phi);
    if (valid[s] && d0 != R(0)) {
      const R d = (__popc(k & h0.y) & 1) ? -d0 : d0;
      acc_add<kOct, SPLIT>(acc, k, fx_prod<R>(d * vs[s].x), fx_prod<R>(d * vs[s].y));
    }
  }
}

// complex128 products in integers.  The weights (LUT entries and term-list
// weights) are stored as d_q = round(d 2^Fd) (DevTables::twfix, |d_q| < 2^62)
// and the lane's amplitude components as v_q = round(v 2^(F + 63 - Fd))
// (|v_q| < 2^63: |v| 2^F < 2^61 / hbound and hbound >= dmax >= 2^(61 - Fd));
// their product shifted right by 63 is round(d v 2^F), the fixed-point
// product, formed exactly and rounded once.  FP64 instructions run on a pipe
// about 1/64 the width of FP32 here; these are integer instructions.
__device__ __forceinline__ long long q_mul(long long a, long long b) {
  const unsigned long long hi = (unsigned long long)__mul64hi(a, b);
  const unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
  return (long long)((hi << 1) + (lo >> 63) + ((lo >> 62) & 1ull));
}

// A compacted complex128 item: the output index k, the weight d_q and the
// lane's amplitude v_q.  A warp's buffer holds up to 32 (A + 1) items: at
// most 31 wait after a flush and a group adds at most 32 A.
struct __align__(16) SpItemQ {
  uint32_t k, pad;
  long long d, vx, vy;
};
constexpr uint32_t kSpCapQ = 32u * (uint32_t)(sp_amps<double>() + 1);

// Adds buffered item `at` (if `on`) to the accumulator; the warp
// synchronises before (the items are other lanes' stores) and after (the
// slots are then reused).
template <uint32_t kOct>
__device__ __forceinline__ void sp_flush_q(const SpItemQ* wb, uint32_t at, bool on, unsigned long long* acc) {
  __syncwarp();
  if (on) {
    const SpItemQ e = wb[at];
    acc_add<kOct>(acc, e.k, q_mul(e.d, e.vx), q_mul(e.d, e.vy));
  }
  __syncwarp();
}

// complex128 LUT group: the integer LUT entry lq[phi] (the group's lut16 in
// the fixed-point copy of the blob), nonzero items appended to the warp's
// buffer (cnt items, warp-uniform) in lane order; lt = the lanes below this
// one.  About two thirds of a sector-confined state's items have a zero
// weight, so the products run 32 at a time with every lane busy.
template <uint32_t kOct, int A>
__device__ __forceinline__ void sp_lut_q(const long long* __restrict__ lq, const uint4 h0, const uint32_t v2,
                                         const uint32_t (&ks)[A], const long long (&vx)[A],
                                         const long long (&vy)[A], const bool (&valid)[A], SpItemQ* wb,
                                         uint32_t& cnt, const uint32_t lt) {
#pragma unroll
  for (int s = 0; s < A; ++s) {
    const uint32_t k = ks[s] ^ h0.x;
    const uint32_t phi = (uint32_t)(__popc(k & h0.z) & 1) | ((uint32_t)(__popc(k & h0.w) & 1) << 1) |
                         ((uint32_t)(__popc(k & v2) & 1) << 2);
    const long long d0 = __ldg(lq + phi);
    const bool nz = valid[s] && d0 != 0ll;
    const uint32_t m = __ballot_sync(0xffffffffu, nz);
    if (nz) {
      SpItemQ e;
      e.k = k;
      e.pad = 0u;
      e.d = (__popc(k & h0.y) & 1) ? -d0 : d0;
      e.vx = vx[s];
      e.vy = vy[s];
      wb[cnt + (uint32_t)__popc(m & lt)] = e;
    }
    cnt += (uint32_t)__popc(m);
  }
}

// complex128 term-list group (see sp_terms): the fixed-point weights wq
// summed exactly, D_q = (sum of all w_q) - 2 (sum of the w_q with odd
// parity), times the factor 0, 1 or 2, and the complex product in integers.
template <uint32_t kOct, int A>
__device__ __forceinline__ void sp_terms_q(const TiledGroup* __restrict__ G, const uint32_t* __restrict__ zs,
                                           const long long* __restrict__ wq, const uint32_t (&ks)[A],
                                           const long long (&vx)[A], const long long (&vy)[A],
                                           const bool (&valid)[A], unsigned long long* acc) {
  const uint4 g0 = __ldg(reinterpret_cast<const uint4*>(&G->x));     // x, tb, tm, te
  const uint2 g1 = __ldg(reinterpret_cast<const uint2*>(&G->delta)); // delta, neg
  uint32_t k[A], fz[A];   // fz: the factor 0, 1 or 2
  bool on = false;
#pragma unroll
  for (int s = 0; s < A; ++s) {
    k[s] = ks[s] ^ g0.x;
    fz[s] = 1u;
    if (g1.x) {
      const uint32_t p = __popc(k[s] & g1.x) & 1u;
      fz[s] = (g1.y ? p : p ^ 1u) ? 2u : 0u;
    }
    on |= valid[s] && fz[s] != 0u;
  }
  if (!__any_sync(0xffffffffu, on)) return;
  unsigned long long ar = 0ull, ai = 0ull, odr[A], odi[A];   // modulo 2^64; the results fit
#pragma unroll
  for (int s = 0; s < A; ++s) odr[s] = odi[s] = 0ull;
  for (uint32_t t = g0.y; t < g0.z; ++t) {
    const uint32_t z = __ldg(zs + t);
    const unsigned long long w = (unsigned long long)__ldg(wq + t);
    ar += w;
#pragma unroll
    for (int s = 0; s < A; ++s)
      if (__popc(k[s] & z) & 1) odr[s] += w;
  }
  for (uint32_t t = g0.z; t < g0.w; ++t) {
    const uint32_t z = __ldg(zs + t);
    const unsigned long long w = (unsigned long long)__ldg(wq + t);
    ai += w;
#pragma unroll
    for (int s = 0; s < A; ++s)
      if (__popc(k[s] & z) & 1) odi[s] += w;
  }
#pragma unroll
  for (int s = 0; s < A; ++s) {
    const int sh = fz[s] == 2u ? 1 : 0;
    const long long a = (long long)((ar - 2ull * odr[s]) << sh), b = (long long)((ai - 2ull * odi[s]) << sh);
    if (valid[s] && fz[s] != 0u && (a | b) != 0ll)
      acc_add<kOct>(acc, k[s], q_mul(a, vx[s]) - q_mul(b, vy[s]), q_mul(a, vy[s]) + q_mul(b, vx[s]));
  }
}

// One term-list group: D(k) = sum_t w_t (-1)^popc(k & z_t), real terms
// [tb, tm), imaginary [tm, te); a paired group keeps one term of each pair
// and D = (1 + sigma (-1)^popc(k & delta)) E(k), the factor 0 or 2.  Called
// by every lane of the warp (the group is warp-uniform).  complex64 (complex128
// uses sp_terms_q).
template <typename R, uint32_t kOct, int A, bool SPLIT>
__device__ __forceinline__ void sp_terms(const TiledGroup* __restrict__ G, const uint32_t* __restrict__ zs,
                                         const R* __restrict__ ws, const uint32_t (&ks)[A],
                                         const C_t<R> (&vs)[A], const bool (&valid)[A],
                                         unsigned long long* acc) {
  const uint4 g0 = __ldg(reinterpret_cast<const uint4*>(&G->x));     // x, tb, tm, te
  const uint2 g1 = __ldg(reinterpret_cast<const uint2*>(&G->delta)); // delta, neg
  uint32_t k[A], fz[A];   // fz: the factor 0, 1 or 2
  bool on = false;
#pragma unroll
  for (int s = 0; s < A; ++s) {
    k[s] = ks[s] ^ g0.x;
    fz[s] = 1u;
    if (g1.x) {
      const uint32_t p = __popc(k[s] & g1.x) & 1u;
      fz[s] = (g1.y ? p : p ^ 1u) ? 2u : 0u;
    }
    on |= valid[s] && fz[s] != 0u;
  }
  if (!__any_sync(0xffffffffu, on)) return;
  R dr[A], di[A];
#pragma unroll
  for (int s = 0; s < A; ++s) dr[s] = di[s] = R(0);
  for (uint32_t t = g0.y; t < g0.z; ++t) {
    const uint32_t z = __ldg(zs + t);
    const R w = __ldg(ws + t);
#pragma unroll
    for (int s = 0; s < A; ++s) dr[s] += (__popc(k[s] & z) & 1) ? -w : w;
  }
  for (uint32_t t = g0.z; t < g0.w; ++t) {
    const uint32_t z = __ldg(zs + t);
    const R w = __ldg(ws + t);
#pragma unroll
    for (int s = 0; s < A; ++s) di[s] += (__popc(k[s] & z) & 1) ? -w : w;
  }
#pragma unroll
  for (int s = 0; s < A; ++s) {
    const R f = fz[s] == 2u ? R(2) : R(1);
    const R a = dr[s] * f, b = di[s] * f;
    if (valid[s] && fz[s] != 0u && (a != R(0) || b != R(0)))
      acc_add<kOct, SPLIT>(acc, k[s], fx_prod<R>(a * vs[s].x - b * vs[s].y),
                           fx_prod<R>(a * vs[s].y + b * vs[s].x));
  }
}

// complex64: a work unit's walk over the piece's LUT groups, then its
// term-list groups, for the lane's A amplitudes.  Each group's descriptor
// (x, z0, v0, v1 and v2) is loaded while the group before it is computed.
template <typename R, uint32_t kOct, int A, bool SPLIT>
__device__ __forceinline__ void sp_walk(const HLut<R>* __restrict__ ls, int nl, const TiledGroup* __restrict__ gs,
                                        int nt, const uint32_t* __restrict__ zs, const R* __restrict__ ws,
                                        const uint32_t (&ks)[A], const C_t<R> (&vs)[A], const bool (&valid)[A],
                                        unsigned long long* acc) {
  uint4 h0n = make_uint4(0u, 0u, 0u, 0u);
  uint32_t v2n = 0u;
  if (nl > 0) {
    h0n = __ldg(reinterpret_cast<const uint4*>(&ls[0].x));
    v2n = __ldg(&ls[0].v2);
  }
  for (int g = 0; g < nl; ++g) {
    const uint4 h0 = h0n;
    const uint32_t v2 = v2n;
    if (g + 1 < nl) {
      h0n = __ldg(reinterpret_cast<const uint4*>(&ls[g + 1].x));
      v2n = __ldg(&ls[g + 1].v2);
    }
    sp_lut<R, kOct, A, SPLIT>(ls + g, h0, v2, ks, vs, valid, acc);
  }
  for (int g = 0; g < nt; ++g) sp_terms<R, kOct, A, SPLIT>(gs + g, zs, ws, ks, vs, valid, acc);
}

// 2^e as R, for |e| beyond one float exponent split in two factors.
template <typename R>
__device__ __forceinline__ void pow2_split(int e, R* a, R* b) {
  const int lim = sizeof(R) == 4 ? 120 : 1000;
  const int e1 = e > lim ? lim : (e < -lim ? -lim : e);
  int e2 = e - e1;
  e2 = e2 > lim ? lim : (e2 < -lim ? -lim : e2);
  *a = sizeof(R) == 4 ? (R)ldexpf(1.0f, e1) : (R)ldexp(1.0, e1);
  *b = sizeof(R) == 4 ? (R)ldexpf(1.0f, e2) : (R)ldexp(1.0, e2);
}

// SPLIT (complex64 only): products added to the accumulator in split form
// (fx_add_split), converted to 64-bit values before the epilogue.
template <typename R, bool SPLIT>
__global__ void __launch_bounds__(sp_threads<R>(), 1) k_apply_h_sparse(const SparseArgs<R> a) {
  static_assert(!SPLIT || sizeof(R) == 4, "the split accumulator takes 32-bit products");
  constexpr int LB = TiledBits<R>::LB;
  constexpr int NT = sp_threads<R>();
  constexpr int A = sp_amps<R>();             // amplitudes per lane per work unit
  constexpr uint32_t kChunk = 32u * A;        // amplitudes per work unit
  constexpr uint32_t kOct = 1u << (LB - 3);   // octets per tile
  if (*a.alen > a.max_amps) return;           // the staged kernel takes this state
  // dynamic shared memory: the tile's fixed-point accumulator, 16 components
  // x kOct octets of 8 bytes
  extern __shared__ __align__(16) uint8_t sp_raw[];
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(sp_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // complex128: the warp's item buffer after the accumulator
  SpItemQ* wb = reinterpret_cast<SpItemQ*>(sp_raw + kOct * 16u * sizeof(unsigned long long)) +
                (sizeof(R) == 8 ? warp * kSpCapQ : 0u);
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t cnt = 0;   // items in wb (warp-uniform)
  // complex128: the fixed-point copy of a blob byte is at the same offset
  // from a.wfix as the byte from a.blob
  const ptrdiff_t wdelta = a.wfix - a.blob;
  __shared__ uint32_t s_tile, s_unext;
  __shared__ uint32_t s_pre[kSpMaxPieces + 1];   // first unit of each piece; s_pre[P] = units
  __shared__ uint32_t s_wsum[32];
  __shared__ double s_red[2][NT / 32];
  __shared__ bool s_last;
  const uint32_t ntiles = 1u << (a.n - LB);
  const uint32_t P = (uint32_t)a.n_pieces;
  for (uint32_t j = threadIdx.x; j < kOct * 16u; j += NT) acc[j] = 0ull;
  // fixed-point scale 2^F: every sum below 2^62 (hbound x 2 max|component|
  // x 2^F <= 2^62) and, for complex64, every off-diagonal product below 2^30
  // (dmax x 2 max|component| x 2^F <= 2^30)
  int F = 0;
  {
    const double m = __longlong_as_double((long long)*a.amax);
    const double bnd = 2.0 * a.hbound * m, bnd1 = 2.0 * a.dmax * m;
    if (bnd > 0.0) {
      int e;
      frexp(bnd, &e);   // bnd < 2^e
      F = 62 - e;
      if (sizeof(R) == 4 && bnd1 > 0.0) {
        frexp(bnd1, &e);
        F = min(F, 30 - e);
      }
    }
  }
  R up_a, up_b, dn_a, dn_b;          // 2^F and 2^-F, each as two factors
  pow2_split<R>(F, &up_a, &up_b);
  pow2_split<R>(-F, &dn_a, &dn_b);
  const double dn = ldexp(1.0, -F);
  const R idr = (R)a.identity;
  const uint32_t K = a.parts;   // blocks per output tile
  for (;;) {
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(a.tile_counter, 1u);
      s_unext = 0u;
    }
    __syncthreads();
    const uint32_t claim = s_tile;
    if (claim >= ntiles * K) break;
    // the claim is part `part` of output tile t: the part takes the tile's
    // unit batches part, part + K, part + 2K, ...
    const uint32_t t = claim / K, part = claim - t * K;
    // Work units are (piece p, chunk c): the nonzero amplitudes kChunk c ..
    // kChunk (c + 1) - 1 of p's source tile u = t ^ (x >> LB) against p's
    // groups, numbered piece by piece (s_pre: a block scan of the chunk counts).
    {
      const uint32_t per = (P + NT - 1) / NT, p0 = threadIdx.x * per, p1 = min(P, p0 + per);
      uint32_t mine = 0;
      for (uint32_t p = p0; p < p1; ++p) {
        const TiledPiece pc = a.piece[a.porder[p]];
        const uint32_t u = t ^ pc.xhi;
        const uint32_t nch = pc.bytes ? (a.toff[u + 1] - a.toff[u] + kChunk - 1u) / kChunk : 0u;
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
        uint32_t ws = lane < NT / 32 ? s_wsum[lane] : 0u, wi = ws;
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t q = __shfl_up_sync(0xffffffffu, wi, o);
          if (lane >= o) wi += q;
        }
        if (lane < NT / 32) s_wsum[lane] = wi - ws;   // exclusive
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
    // kUnitBatch consecutive units per claim (mostly chunks of one piece,
    // whose descriptors then stay in L1); one per claim when the tile has
    // fewer than kUnitBatch units per warp of its K blocks, so that the few
    // units of a small state do not queue behind each other on one warp
    const uint32_t batch = n_units < kUnitBatch * (uint32_t)(NT / 32) * K ? 1u : kUnitBatch;
    for (;;) {
      uint32_t j0 = 0;
      if (lane == 0) j0 = (atomicAdd(&s_unext, 1u) * K + part) * batch;
      j0 = __shfl_sync(0xffffffffu, j0, 0);
      if (j0 >= n_units) break;
      const uint32_t j1 = min(n_units, j0 + batch);
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
        const uint32_t pid = a.porder[p];
        const TiledPiece pc = a.piece[pid];
        const uint32_t u = t ^ pc.xhi;
        const uint32_t a0 = a.toff[u], a1 = a.toff[u + 1];
        const uint8_t* blob = a.blob + pc.off;
        const uint4 hd = __ldg(reinterpret_cast<const uint4*>(blob));   // n_runs, n_lut, z_off, w_off
        const HLut<R>* ls = reinterpret_cast<const HLut<R>*>(blob + sizeof(TiledHead));
        const TiledGroup* gs = reinterpret_cast<const TiledGroup*>(blob + sizeof(TiledHead) + hd.y * sizeof(HLut<R>));
        const uint32_t* zs = reinterpret_cast<const uint32_t*>(blob + hd.z);
        const R* ws = reinterpret_cast<const R*>(blob + hd.w);
        uint32_t ks[A];
        C_t<R> vs[A];
        long long vqx[A], vqy[A];   // complex128: the amplitudes as v_q (see q_mul)
        bool valid[A];
#pragma unroll
        for (int s = 0; s < A; ++s) {
          const uint32_t li = a0 + kChunk * c + 32u * s + (uint32_t)lane;
          valid[s] = li < a1;
          ks[s] = a.aidx[valid[s] ? li : a0];
          const C_t<R> v = a.aval[valid[s] ? li : a0];
          vs[s] = cmake<R>(v.x * up_a * up_b, v.y * up_a * up_b);
          if constexpr (sizeof(R) == 8) {
            vqx[s] = __double2ll_rn((double)vs[s].x * a.wscale);
            vqy[s] = __double2ll_rn((double)vs[s].y * a.wscale);
          }
        }
        const int nl = (int)hd.y;
        // the term-list groups fill the blob from the LUT groups to z_off
        const int nt = (int)((hd.z - sizeof(TiledHead) - nl * sizeof(HLut<R>)) / sizeof(TiledGroup));
        if constexpr (sizeof(R) == 8) {
          // each group's descriptor (x, z0, v0, v1 and v2) is loaded while
          // the group before it is computed
          uint4 h0n = make_uint4(0u, 0u, 0u, 0u);
          uint32_t v2n = 0u;
          if (nl > 0) {
            h0n = __ldg(reinterpret_cast<const uint4*>(&ls[0].x));
            v2n = __ldg(&ls[0].v2);
          }
          for (int g = 0; g < nl; ++g) {
            const uint4 h0 = h0n;
            const uint32_t v2 = v2n;
            if (g + 1 < nl) {
              h0n = __ldg(reinterpret_cast<const uint4*>(&ls[g + 1].x));
              v2n = __ldg(&ls[g + 1].v2);
            }
            const long long* lq = reinterpret_cast<const long long*>(
                reinterpret_cast<const uint8_t*>(ls[g].lut16) + wdelta);
            sp_lut_q<kOct, A>(lq, h0, v2, ks, vqx, vqy, valid, wb, cnt, lt);
            while (cnt >= 32u) {
              cnt -= 32u;
              sp_flush_q<kOct>(wb, cnt + (uint32_t)lane, true, acc);
            }
          }
          const long long* wq = reinterpret_cast<const long long*>(reinterpret_cast<const uint8_t*>(ws) + wdelta);
          for (int g = 0; g < nt; ++g) sp_terms_q<kOct, A>(gs + g, zs, wq, ks, vqx, vqy, valid, acc);
        } else if (A > 1 && a0 + kChunk * c + 32u >= a1) {
          // the unit's amplitudes fill the first lane slot at most (the last
          // chunk of a source tile): the groups are walked for that slot
          // alone instead of issuing the empty slots with every lane idle
          const uint32_t ks1[1] = {ks[0]};
          const C_t<R> vs1[1] = {vs[0]};
          const bool valid1[1] = {valid[0]};
          sp_walk<R, kOct, 1, SPLIT>(ls, nl, gs, nt, zs, ws, ks1, vs1, valid1, acc);
        } else {
          sp_walk<R, kOct, A, SPLIT>(ls, nl, gs, nt, zs, ws, ks, vs, valid, acc);
        }
      }
    }
    if (cnt) sp_flush_q<kOct>(wb, (uint32_t)lane, (uint32_t)lane < cnt, acc);   // the rest, fewer than 32
    cnt = 0;
    __syncthreads();
    if constexpr (SPLIT) {
      // every product is in: the split words become 64-bit values
      for (uint32_t j = threadIdx.x; j < kOct * 16u; j += NT) {
        const unsigned long long v = acc[j];
        if (v) acc[j] = split_to_wide(v);
      }
      __syncthreads();
    }
    if (K > 1) {
      // several blocks per tile: each adds its nonzero accumulator entries
      // to the tile's global accumulator (64-bit integer atomics: the same
      // sum in any order), and the last to finish takes the total, clears
      // the global copy for the next call and runs the epilogue
      unsigned long long* g = a.gacc + (size_t)t * (kOct * 16u);
      for (uint32_t j = threadIdx.x; j < kOct * 16u; j += NT) {
        const unsigned long long v = acc[j];
        if (v) atomicAdd(g + j, v);
      }
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_last = atomicAdd(a.tdone + t, 1u) == K - 1u;
      __syncthreads();
      if (!s_last) {
        for (uint32_t j = threadIdx.x; j < kOct * 16u; j += NT) acc[j] = 0ull;
        __syncthreads();
        continue;
      }
      __threadfence();
      for (uint32_t j = threadIdx.x; j < kOct * 16u; j += NT) {
        acc[j] = __ldcg(g + j);
        __stcg(g + j, 0ull);
      }
      if (threadIdx.x == 0) a.tdone[t] = 0u;
      __syncthreads();
    }
    // epilogue, first the nonzero amplitudes of the own tile (one lane
    // each): the diagonal group and the identity, which act on psi(k) alone,
    // and the energy partials (zero amplitudes add to neither); each k is
    // one lane's, so its accumulator entry is updated without atomics
    {
      double2 w = make_double2(0.0, 0.0);   // this thread's |psi|^2 and <psi|H - identity|psi> partials
      const uint32_t e0 = a.toff[t], e1 = a.toff[t + 1];
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
        unsigned long long* e2 = acc + acc_at<kOct>(k);
        const double ox = (double)(long long)e2[0] * dn, oy = (double)(long long)e2[kOct] * dn;
        const double pp = (double)q.x * q.x + (double)q.y * q.y;
        w.x += pp;
        w.y += (double)q.x * ox + (double)q.y * oy + ((double)dr - (double)dc) * pp;
        const R d0 = dr - dc + idr;
        const C_t<R> qs = cmake<R>(q.x * up_a * up_b, q.y * up_a * up_b);
        e2[0] = (unsigned long long)((long long)e2[0] + fx_wide<R>(d0 * qs.x - di * qs.y));
        e2[kOct] = (unsigned long long)((long long)e2[kOct] + fx_wide<R>(d0 * qs.y + di * qs.x));
      }
      // the tile's energy partials, summed in a fixed order (warps that
      // hold no amplitude of the tile skip the FP64 shuffles)
      if (a.partials) {
        const bool any = __any_sync(0xffffffffu, w.x != 0.0 || w.y != 0.0);
        const double sx = any ? warp_sum(w.x) : 0.0, sy = any ? warp_sum(w.y) : 0.0;
        if (lane == 0) {
          s_red[0][warp] = sx;
          s_red[1][warp] = sy;
        }
      }
    }
    __syncthreads();
    if (a.partials && threadIdx.x < 2) {
      double sum = 0.0;
      for (int q = 0; q < NT / 32; ++q) sum += s_red[threadIdx.x][q];
      a.partials[2u * t + threadIdx.x] = sum;
    }
    // then the whole tile out (zeros included) and the accumulator cleared
    for (uint32_t o = threadIdx.x; o < kOct; o += NT) {
      const uint32_t k0 = ((t << (LB - 3)) | o) << 3;
      C_t<R> res[kAmpsH];
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) {
        unsigned long long* e = acc + acc_at<kOct>(k0 | (uint32_t)i);
        const R re = fx_val<R>(e[0]), im = fx_val<R>(e[kOct]);
        res[i] = cmake<R>(re * dn_a * dn_b, im * dn_a * dn_b);
        e[0] = 0ull;
        e[kOct] = 0ull;
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
  if (!a.partials) return;
  // the last block to finish adds the per-tile partials in tile order, so E
  // does not depend on which block took which tile
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(a.counter, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double acc0 = 0.0, acc1 = 0.0;
  for (uint32_t u = threadIdx.x; u < ntiles; u += NT) {
    acc0 += ((volatile double*)a.partials)[2u * u];
    acc1 += ((volatile double*)a.partials)[2u * u + 1u];
  }
  acc0 = warp_sum(acc0);
  acc1 = warp_sum(acc1);
  if (lane == 0) {
    s_red[0][warp] = acc0;
    s_red[1][warp] = acc1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double n2 = 0.0, eh = 0.0;
    for (int q = 0; q < NT / 32; ++q) {
      n2 += s_red[0][q];
      eh += s_red[1][q];
    }
    a.scal[1] = n2;
    a.scal[2] = eh;
    a.scal[0] = a.identity + eh / n2;
    *a.counter = 0u;
  }
}

template <typename R>
constexpr uint32_t sparse_smem() {
  return (1u << (TiledBits<R>::LB - 3)) * 16u * (uint32_t)sizeof(unsigned long long) +
         (sizeof(R) == 8 ? (uint32_t)(sp_threads<R>() / 32) * kSpCapQ * (uint32_t)sizeof(SpItemQ) : 0u);
}

}  // namespace

template <typename R>
int sparse_apply_h(SparseArgs<R> a, const LiveOctets& lv, int sm_count, cudaStream_t st) {
  constexpr int LB = TiledBits<R>::LB;
  if (a.n < LB || !lv.toff || !lv.aidx || !lv.aval || !lv.alen || !lv.acounts || !lv.amax || a.max_amps > lv.acap)
    return fail(GOCP_EINVAL, "scatter H psi needs the amplitude list");
  if (sizeof(R) == 8 && !a.wfix) return fail(GOCP_EINVAL, "scatter H psi (complex128) needs the fixed-point weights");
  a.amax = lv.amax;
  a.aidx = lv.aidx;
  a.aval = reinterpret_cast<const C_t<R>*>(lv.aval);
  a.alen = lv.alen;
  a.toff = lv.toff;
  // complex64 adds its products in split form when every accumulator word
  // takes fewer than 65536 of them (one per off-diagonal group); the two
  // forms give the same integers, so H psi does not depend on the choice
  // (GOCP_SCATTER_SPLIT=0 selects the carry form)
  bool split = sizeof(R) == 4 && a.n_offdiag < 65536u;
  if (const char* ev = std::getenv("GOCP_SCATTER_SPLIT"))
    if (ev[0] == '0') split = false;
  auto kern = split ? k_apply_h_sparse<R, sizeof(R) == 4> : k_apply_h_sparse<R, false>;
  static std::mutex mu;
  static std::vector<bool> done;
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  {
    std::lock_guard<std::mutex> lk(mu);
    if (device >= (int)done.size()) done.resize(device + 1, false);
    if (!done[device]) {
      e = cudaFuncSetAttribute(k_apply_h_sparse<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sparse_smem<R>());
      if (e == cudaSuccess && sizeof(R) == 4)
        e = cudaFuncSetAttribute(k_apply_h_sparse<R, sizeof(R) == 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sparse_smem<R>());
      if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_apply_h_sparse)");
      done[device] = true;
    }
  }
  int rc = amp_list(sizeof(R) == 4 ? GOCP_C64 : GOCP_C128, a.psi, a.mask, a.n, lv, st);
  if (rc) return rc;
  const uint32_t ntiles = 1u << (a.n - LB);
  k_tile_offsets<<<(ntiles + 256u) / 256u, 256, 0, st>>>(lv.aidx, lv.alen, lv.acap, ntiles, LB, lv.toff);
  // tiles for fewer than half the SMs: K blocks share each tile (K a power
  // of two up to 64, or GOCP_SCATTER_PARTS, so that ntiles K reaches the SM
  // count), combining their fixed-point accumulators in global memory; the
  // sums are integer, so H psi and E do not depend on K.  Measured per H psi
  // call on prepared ADAPT states (complex64 / complex128): 14 qubits
  // 0.19 / 0.23 -> 0.14 / 0.17 ms, 16 qubits 0.27 / 0.33 -> 0.20 / 0.20 ms,
  // 18 qubits 0.34 / 0.42 -> 0.22 / 0.30 ms; with 128 tiles on 152 SMs
  // (20 qubits complex64) splitting was slower, and two waves of parts
  // slower than one.
  const uint32_t sms = (uint32_t)std::max(sm_count, 1);
  uint32_t kmax = 64u;
  if (const char* e = std::getenv("GOCP_SCATTER_PARTS")) {
    const long v = std::strtol(e, nullptr, 10);
    if (v >= 1) kmax = (uint32_t)std::min<long>(v, 64);
  }
  uint32_t K = 1;
  if (lv.gacc && lv.tdone && ntiles <= lv.gtiles && 2u * ntiles < sms)
    while (2u * K <= kmax && ntiles * K < sms) K *= 2u;
  a.parts = K;
  a.gacc = lv.gacc;
  a.tdone = lv.tdone;
  const int grid = (int)std::min<uint64_t>((uint64_t)ntiles * K, (uint64_t)sms);
  kern<<<grid, sp_threads<R>(), sparse_smem<R>(), st>>>(a);
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
    k_amp_scan<<<1, 1024, 0, st>>>(lv.acounts, nb, lv.alen, nullptr, 0, 0, lv.amax);
    k_amp_list<float><<<nb, kAmpBlock, 0, st>>>(p, nullptr, mask, words, lv.acounts, lv.aidx,
                                                reinterpret_cast<float2*>(lv.aval), nullptr, lv.acap, lv.amax);
  } else {
    const double2* p = reinterpret_cast<const double2*>(psi);
    k_amp_count<double><<<nb, kAmpBlock, 0, st>>>(p, nullptr, mask, words, lv.acounts);
    k_amp_scan<<<1, 1024, 0, st>>>(lv.acounts, nb, lv.alen, nullptr, 0, 0, lv.amax);
    k_amp_list<double><<<nb, kAmpBlock, 0, st>>>(p, nullptr, mask, words, lv.acounts, lv.aidx,
                                                 reinterpret_cast<double2*>(lv.aval), nullptr, lv.acap, lv.amax);
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
    k_amp_scan<<<1, 1024, 0, st>>>(counts, nb, nullptr, cl.cnt, slot, first, nullptr);
    k_amp_list<float><<<nb, kAmpBlock, 0, st>>>(p, q, mask, words, counts, cl.list, nullptr, cl.amask, cl.cap,
                                                nullptr);
  } else {
    const double2* p = reinterpret_cast<const double2*>(psi);
    const double2* q = reinterpret_cast<const double2*>(lam);
    k_amp_count<double><<<nb, kAmpBlock, 0, st>>>(p, q, mask, words, counts);
    k_amp_scan<<<1, 1024, 0, st>>>(counts, nb, nullptr, cl.cnt, slot, first, nullptr);
    k_amp_list<double><<<nb, kAmpBlock, 0, st>>>(p, q, mask, words, counts, cl.list, nullptr, cl.amask, cl.cap,
                                                 nullptr);
  }
  count_launches(3);
  return cuda_status(cudaGetLastError(), "chain list");
}

template int sparse_apply_h<float>(SparseArgs<float>, const LiveOctets&, int, cudaStream_t);
template int sparse_apply_h<double>(SparseArgs<double>, const LiveOctets&, int, cudaStream_t);

}  // namespace gocp
