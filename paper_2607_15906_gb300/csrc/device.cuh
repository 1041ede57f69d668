// Device-side types shared by the kernels and their launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace gocp {

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

template <typename R> using C_t = typename Cplx<R>::T;

template <typename R>
__host__ __device__ __forceinline__ C_t<R> cmake(R re, R im) {
  C_t<R> v;
  v.x = re;
  v.y = im;
  return v;
}
template <typename R>
__device__ __forceinline__ C_t<R> cadd(C_t<R> a, C_t<R> b) { return cmake<R>(a.x + b.x, a.y + b.y); }
template <typename R>
__device__ __forceinline__ C_t<R> csub(C_t<R> a, C_t<R> b) { return cmake<R>(a.x - b.x, a.y - b.y); }
template <typename R>
__device__ __forceinline__ C_t<R> cmul(C_t<R> a, C_t<R> b) {
  return cmake<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
__device__ __forceinline__ C_t<R> cscale(C_t<R> a, R s) { return cmake<R>(a.x * s, a.y * s); }
template <typename R>
__device__ __forceinline__ C_t<R> cconj(C_t<R> a) { return cmake<R>(a.x, -a.y); }

// v == 0 (either sign of zero).  For double the test is on the bits, with
// integer instructions: FP64 compares run on the FP64 pipe, about 1/64 the
// width of FP32 on this part.
template <typename R>
__device__ __forceinline__ bool rzero(R v) {
  if constexpr (sizeof(R) == 8) return (__double_as_longlong((double)v) << 1) == 0ll;
  else return v == R(0);
}

// Start of one step of a chain launched with programmatic dependencies
// (launch_chain): wait until the previous step's grid has finished and its
// writes are visible, then let the next step's blocks be scheduled while this
// one runs.  Both instructions do nothing in a kernel launched without such a
// dependency.
__device__ __forceinline__ void chain_step_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// An x-group (or generator) in LUT form, see LutForm:
//   D(b) = (-1)^popc(b & z0) * lut[phi(b)],  phi(b) = sum_i (popc(b & v_i) & 1) << i,
// with real weights only.  fx holds phi(x) (bits 0..2) and popc(x & z0) & 1
// (bit 3), so that D(b ^ x) = (-1)^(sigma(b) ^ bit3) * lut[phi(b) ^ phi(x)].
// s is the lowest set bit of x (the pivot that enumerates pairs {b, b^x}).
// An exactly zero lut entry means the operator does not touch those basis
// states: kernels skip them without changing any result.
template <typename R>
struct LutDev {
  uint32_t x, z0, v0, v1, v2;
  uint32_t fx;
  int32_t s;
  int32_t pad;
  R lut[8];
};

template <typename R>
__device__ __forceinline__ uint32_t lut_phi(const LutDev<R>& L, uint32_t b) {
  return (uint32_t)(__popc(b & L.v0) & 1) | ((uint32_t)(__popc(b & L.v1) & 1) << 1) |
         ((uint32_t)(__popc(b & L.v2) & 1) << 2);
}

// The basis pairs {b, b^x} (b with bit s clear) that a LUT-form generator
// touches, i.e. lut[phi(b)] != 0 or lut[phi(b) ^ phi(x)] != 0, as an
// enumerable set: for each touched code, b is a counter deposited into the
// free bit positions (all but s and the r pivot positions, `excl`, ascending)
// with pivot bit k set to the reduced code bit k xor popc(b & pmask[k]).
// codes: byte j = reduced code (bits 0..2) | original code << 3 of the j-th
// touched code.  count = ncodes << log2cnt pairs.
struct PairEnum {
  uint32_t excl;       // nex positions, one per byte, ascending
  uint32_t piv;        // r pivot positions, one per byte
  uint32_t pmask[3];
  uint32_t codes;      // up to 4 touched codes (generators of rank <= 3 touch at most 4)
  uint32_t codes_hi;   // codes 4..7
  uint8_t nex, r, ncodes, log2cnt;
};

__device__ __forceinline__ uint32_t enum_deposit(uint32_t c, uint32_t excl, int nex) {
  for (int e = 0; e < nex; ++e) {
    const uint32_t p = (excl >> (8 * e)) & 0xFFu;
    c = ((c >> p) << (p + 1)) | (c & ((1u << p) - 1u));
  }
  return c;
}

// Pair base b and original code of enumerated pair `idx`.
__device__ __forceinline__ uint32_t enum_pair(const PairEnum& e, uint32_t idx, uint32_t* code) {
  const uint32_t ci = idx >> e.log2cnt;
  const uint32_t cnt = idx & ((1u << e.log2cnt) - 1u);
  const uint32_t byte = ((ci < 4 ? e.codes : e.codes_hi) >> (8 * (ci & 3))) & 0xFFu;
  uint32_t b = enum_deposit(cnt, e.excl, e.nex);
  const uint32_t bf = b;
  for (int k = 0; k < e.r; ++k) {
    const uint32_t bit = ((byte >> k) & 1u) ^ (uint32_t)(__popc(bf & e.pmask[k]) & 1);
    b |= bit << ((e.piv >> (8 * k)) & 0xFFu);
  }
  *code = byte >> 3;
  return b;
}

// An H x-group in LUT form for the H psi kernel, whose threads own 8
// adjacent amplitudes k0 + i (k0 a multiple of 8): code(k) = phi(k) | sigma(k) << 3
// with sigma(k) = popc(k & z0) & 1, so that D(k) = lut16[code(k)] (the sign
// is folded into the table) and code(k0 + i) = code(k0) ^ ((reg >> 4i) & 15).
template <typename R>
struct __align__(16) HLut {
  uint32_t x, z0, v0, v1;   // read as one 16-byte vector
  uint32_t v2, reg;         // and one 8-byte vector
  uint32_t pad0, pad1;
  R lut16[16];
};

// H psi by shared-memory tiles (apply_tiled.cu).  A tile is 2^LB amplitudes
// (64 KiB: LB = 13 for complex64, 12 for complex128); the groups are cut into
// pieces by their high mask bits x >> LB, so that every group of a piece
// reads the same source tile.  A piece is a contiguous blob, copied to shared
// memory in one bulk copy beside its source tile:
//   TiledHead | HLut<R>[n_lut] | TiledGroup[n_tg] | z[] | w[]
// with the LUT groups sorted by (flip class, x & 7, x), the term-list groups
// by (x & 7, x), each list cut into runs of one kernel variant.  The pieces of
// one high pattern follow each other; the pieces with x >> LB = 0 come last
// (there is always one), so that the own tile is staged for the diagonal.
#ifndef GOCP_TILED_LB_C64
#define GOCP_TILED_LB_C64 13
#endif
template <typename R> struct TiledBits;
template <> struct TiledBits<float> { static constexpr int LB = GOCP_TILED_LB_C64; };
template <> struct TiledBits<double> { static constexpr int LB = 12; };
constexpr uint32_t kTiledBlobBytes = 4096;    // largest piece blob

constexpr int kTiledRuns = 32;   // runs per piece
struct TiledHead {
  uint32_t n_runs, n_lut;
  uint32_t z_off, w_off;        // byte offsets of the term arrays in the blob
  // the non-empty runs: begin (bits 0..11) and end (12..23) in their list,
  // and a kernel selector (24..30): 8 F + (x & 7) for LUT groups of flip
  // class F (see tiled_flip_class), 64 + (x & 7) for term-list groups
  uint32_t run[kTiledRuns];
};
static_assert(sizeof(TiledHead) == 144, "TiledHead is 144 bytes");

// Flip class of an H LUT group: bit b set when the code of k0 + 2^b differs
// from the code of k0 (nibble 2^b of HLut::reg is nonzero).  The code flip
// of octet member i is the XOR of those of its bits, so member i has the
// same LUT entry as member i & F.
__host__ __device__ __forceinline__ uint32_t tiled_flip_class(uint32_t reg) {
  return (uint32_t)(((reg >> 4) & 15u) != 0u) | ((uint32_t)(((reg >> 8) & 15u) != 0u) << 1) |
         ((uint32_t)(((reg >> 16) & 15u) != 0u) << 2);
}

// A term-list group.  When delta != 0 its terms come in exact pairs
// (z, w), (z ^ delta, sigma w): then D(k) = (1 + sigma (-1)^popc(k & delta)) E(k),
// a factor that is exactly 0 or 2, and only one term of each pair is kept
// (E's terms).  Number-conserving one-body groups have this form.
struct __align__(16) TiledGroup {
  uint32_t x;
  uint32_t tb, tm, te;          // [tb, tm) real, [tm, te) imaginary terms
  uint64_t bk;                  // Walsh bucket sizes (see DevTables::gbk)
  uint32_t xa;                  // tiled_swz<R>((x >> 3) & (octets - 1))
  uint32_t pad;                 // (x >> 3) & (octets - 1)
  uint32_t delta;               // pair vector, 0: unpaired
  uint32_t neg;                 // 1: sigma = -1, 0: sigma = +1
  uint32_t pad2[2];
};
static_assert(sizeof(TiledGroup) == 48, "TiledGroup is 48 bytes");

// Byte offset of octet o in a staged tile.  The tile is rows of 128 bytes
// whose 16-byte chunks sit at chunk ^ (row & 7) (the 128-byte swizzle of the
// tensor copy); chunk q of the octet (amplitudes 2q, 2q+1 for complex64,
// amplitude q for complex128) is at tiled_swz(o) ^ (q << 4).  The map is
// linear over XOR, tiled_swz(o ^ c) = tiled_swz(o) ^ tiled_swz(c), so the
// kernel adds a group's source offset c with one XOR of a value the host
// stores with the group (HLut::pad0, TiledGroup::xa); c itself, which indexes
// the nonzero-octet mask, is stored beside it (HLut::pad1, TiledGroup::pad).
template <typename R>
__host__ __device__ __forceinline__ uint32_t tiled_swz(uint32_t o) {
  return sizeof(R) == 4 ? ((o >> 1) << 7) | ((((o & 1u) << 2) ^ ((o >> 1) & 7u)) << 4)
                        : (o << 7) | ((o & 7u) << 4);
}

// One piece: x >> LB of its groups, byte offset and size of its blob.
struct __align__(16) TiledPiece {
  uint32_t xhi, off, bytes, pad;
};

// Nonzero-amplitude list carried through a tracked chain of Taylor or
// adjoint steps (LUT pools, n >= 8): the first entries of list hold every
// nonzero amplitude index of the chain's state(s) (and possibly indices whose
// amplitude became zero again) and amask has their bits (2^n bits).  The
// list length is kept in a ring of three slots, slot i = step j mod 3: a
// step starts at length base(p) + count(p) (p = the previous step's slot:
// its start + the entries it appended), records that start as its own base,
// appends by counting in its own count, and zeroes the next step's count.
// A length above cap: the list is incomplete and the steps enumerate the
// operator's pairs instead.
// Ring words: slot i's base at cnt[kRingBase(i)], its count at
// cnt[kRingAdd(i)], each in its own 32-byte sector.
__host__ __device__ constexpr int kRingBase(int i) { return 8 * i; }
__host__ __device__ constexpr int kRingAdd(int i) { return 24 + 8 * i; }
constexpr int kRingWords = 48;

struct ChainList {
  uint32_t* list = nullptr;
  uint32_t* amask = nullptr;
  uint32_t* cnt = nullptr;
  uint32_t cap = 0;
};

// Device copies of the tables of one problem.
//
// Hamiltonian: the identity term is a scalar; the diagonal group (x = 0) is
// kept apart; the other groups of terms sharing an x mask come in ascending
// x.  Group g owns
// terms [goff[g], goff[g+1]); terms [goff[g], gmid[g]) have real weights,
// [gmid[g], goff[g+1]) imaginary ones.  The weight of term t is
//   w_t = c_t i^phase_t (-1)^popc(x_g & z_t),
// so that (H psi)[k] = sum_g D_g(k) psi[k ^ x_g] with
//   D_g(k) = sum_{t in g} w_t (-1)^popc(k & z_t).
// chunk_g splits the groups into runs whose terms fit the shared-memory
// stage of the H psi kernel (a run of one group may exceed it).
//
// Pool: generator k owns strings [poff[k], poff[k+1]) with one x mask px[k]
// (real-weight strings first, split at pmid[k]).  pw holds w_t as above and
// pw2 holds w_t (-1)^popc(x & z_t), so that for a basis pair (b, b ^ x) one
// parity per string gives both D(b) and D(b ^ x).  porder lists the pool in
// GOCP family order.
struct DevTables {
  int n = 0;
  int G = 0, n_chunks = 0;
  int64_t T = 0;
  const uint32_t* gx = nullptr;
  const int32_t* goff = nullptr;
  const int32_t* gmid = nullptr;
  const int32_t* chunk_g = nullptr;
  const uint32_t* tz = nullptr;
  const void* tw = nullptr;
  // off-diagonal groups in LUT form (real weights, rank <= 3), ascending x;
  // the term groups above hold the rest
  int GL = 0;
  const void* hlut = nullptr;
  // groups are sorted by x & 7 and split into chunks that never mix two
  // values of x & 7; chunk c of LUT groups is [lchunk[c], lchunk[c+1]) with
  // lchunk_xl[c] = x & 7, and likewise chunk_xl for the term-list chunks
  int n_lchunks = 0;
  const int32_t* lchunk = nullptr;
  const uint8_t* lchunk_xl = nullptr;
  const uint8_t* chunk_xl = nullptr;
  // per term-list group: the real terms are sorted by z & 7 and gbk packs the
  // eight bucket sizes (byte m = terms with z & 7 == m); ~0 when the group
  // has imaginary terms or a bucket above 255 (then it is summed term by term)
  const uint64_t* gbk = nullptr;
  // the tiled form of the off-diagonal groups (n_pieces = 0: none), and
  // (n >= 8) a scratch mask of 2^(n-3) bits over the octets of a state: a
  // clear bit guarantees that the octet's 8 amplitudes are exactly zero (set
  // bits may be conservative); see octet_mask
  int n_pieces = 0;
  const uint8_t* tblob = nullptr;
  const TiledPiece* tpiece = nullptr;
  const uint32_t* tporder = nullptr;   // piece indices by descending blob size
  // complex128: the blobs' LUT entries and term-list weights as 64-bit
  // fixed-point integers round(w 2^Fd), each at its value's offset in tblob
  // (elsewhere zero), Fd = 62 - e with dmax < 2^e; and twscale = 2^(63 - Fd),
  // the factor that takes an amplitude scaled by 2^F to the integer whose
  // product with a weight, shifted right by 63, is the product at 2^F
  const uint8_t* twfix = nullptr;
  double twscale = 0.0;
  uint32_t* octmask = nullptr;
  uint32_t* tflags = nullptr;   // tiled form: one bit per tile (scratch)
  // second mask of the same size, for the adjoint sweep (psi and lambda)
  uint32_t* octmask2 = nullptr;
  // sector layout (see SecDev): per LUT group (hlut order), term-list group
  // and generator (pool order) the occupation-space flip u = beta^-1 x, its
  // alpha string in bits 0..15 and its beta string in bits 16..31; and the
  // term-list groups in paired form where they pair (sp_delta != 0, see
  // TiledGroup), kept terms [sp_off[g], sp_mid[g]) real and
  // [sp_mid[g], sp_off[g + 1]) imaginary in sp_z / sp_w
  const uint32_t* hu = nullptr;
  const uint32_t* gu = nullptr;
  const uint32_t* pu = nullptr;
  const uint32_t* sp_delta = nullptr;
  const uint32_t* sp_neg = nullptr;
  const int32_t* sp_off = nullptr;
  const int32_t* sp_mid = nullptr;
  const uint32_t* sp_z = nullptr;
  const void* sp_w = nullptr;
  // diagonal group (x = 0) without the identity: [0, nd_mid) real, [nd_mid, nd) imaginary
  int nd = 0, nd_mid = 0;
  // bound on the magnitude of H's couplings at any basis state: the sum over
  // the off-diagonal groups of max_k |D_g(k)|, plus the diagonal group's and
  // the identity's sum of |w| (the scatter kernel's fixed-point scale)
  double hbound = 0.0;
  // the largest coupling of one off-diagonal group, max_g max_k |D_g(k)|
  // (term-list groups: the sum of their |w|)
  double dmax = 0.0;
  const uint32_t* dz = nullptr;
  const void* dw = nullptr;
  int M = 0;
  int64_t S = 0;
  const uint32_t* px = nullptr;
  const int32_t* poff = nullptr;
  const int32_t* pmid = nullptr;
  const uint32_t* pz = nullptr;
  const void* pw = nullptr;
  const void* pw2 = nullptr;
  const int32_t* porder = nullptr;
  // every generator in LUT form (pool order), when all of them qualify, and
  // the enumeration of the pairs each one touches
  bool pool_lut = false;
  const void* plut = nullptr;
  const PairEnum* penum = nullptr;
  uint32_t penum_max = 0;   // largest touched-pair count of any generator
  ChainList cl;             // tracked chains (list == nullptr: none)
};


// ------------------------------------------------------------ shared device helpers

// H psi octets: a thread owns kAmpsH = 8 adjacent amplitudes k0 + i (k0 a
// multiple of 8).
constexpr int kAmpsH = 8;
// Walsh sign patterns: byte m holds bit i = popc(i & m) & 1 for i, m < 8
constexpr uint64_t kWalsh8 = 0x963C5AF066CCAA00ull;

// Sign bits (bit i = amplitude k0 + i) of (-1)^popc((k0 + i) & z).
__device__ __forceinline__ uint32_t octet_signs(uint32_t k0, uint32_t z) {
  const uint32_t pat = (uint32_t)(kWalsh8 >> (8 * (z & 7u))) & 0xFFu;
  return pat ^ ((__popc(k0 & z) & 1u) * 0xFFu);
}

// d[i] += sum_{t in [tb, te)} w_t (-1)^popc((k0+i) & z_t); compensated in
// FP32 when asked (comp carries the lost low part: true sum d - comp).
template <typename R>
__device__ __forceinline__ void sum_terms8(const uint32_t* zs, const R* ws, int tb, int te,
                                           uint32_t k0, R (&d)[kAmpsH], R (&comp)[kAmpsH],
                                           bool compensate) {
  if (sizeof(R) == 4 && compensate) {
    for (int t = tb; t < te; ++t) {
      const uint32_t sg = octet_signs(k0, zs[t]);
      const R w = ws[t];
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) {
        R y = (((sg >> i) & 1u) ? -w : w) - comp[i];
        R s = d[i] + y;
        comp[i] = (s - d[i]) - y;
        d[i] = s;
      }
    }
  } else {
    for (int t = tb; t < te; ++t) {
      const uint32_t sg = octet_signs(k0, zs[t]);
      const R w = ws[t];
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) d[i] += ((sg >> i) & 1u) ? -w : w;
    }
  }
}

// ------------------------------------------------------------ reductions

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// c[m] = theta^m / m! of step j in R, converted once per block (FP64 is a
// slow pipe on this part; a conversion in every thread costs microseconds
// per step).  Called by every thread of the block.
template <typename R>
__device__ __forceinline__ void step_coefs(const double* coefs, int j, R (&c)[6]) {
  __shared__ R s_c[6];
  if (threadIdx.x < 6) s_c[threadIdx.x] = (R)coefs[6 * j + threadIdx.x];
  __syncthreads();
#pragma unroll
  for (int m = 0; m < 6; ++m) c[m] = s_c[m];
}

// Sum over the warp in R; the total in lane 0.
template <typename R>
__device__ __forceinline__ R warp_total(R v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Adds v[0..NV) over the nblocks blocks (NTHREADS threads each) of one work
// item into out[0..NV).  WarpReduced: the caller has already summed each
// warp (the total in lane 0, the other lanes ignored), so the FP64 warp
// reduction is skipped.
// partials: NV doubles per block; counter: one per item, zero on entry and
// reset on exit.  Returns true in the last block, where tot[0..NV) (shared)
// then holds the totals for every thread.
template <int NV, int NTHREADS, bool WarpReduced = false>
__device__ bool block_grid_sum(const double (&v)[NV], double* partials, unsigned int* counter,
                               int nblocks, int bid, double* out, double* tot) {
  __shared__ double red[NV][NTHREADS / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = WarpReduced ? v[i] : warp_sum(v[i]);
    if (lane == 0) red[i][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < NTHREADS / 32; ++w) s += red[threadIdx.x][w];
    partials[(size_t)bid * NV + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned)(nblocks - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += NTHREADS) {
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] += ((volatile double*)partials)[(size_t)b * NV + i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = warp_sum(acc[i]);
    if (lane == 0) red[i][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < NTHREADS / 32; ++w) s += red[threadIdx.x][w];
    out[threadIdx.x] = s;
    tot[threadIdx.x] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
  __syncthreads();
  return true;
}

// Rows of the sector layout: the D determinants with na alpha and nb beta
// electrons among no spatial orbitals, row r = rank_a[alpha] * cb +
// rank_b[beta] (colexicographic ranks, cb = C(no, nb)).  An occupation is
// kept as alpha | beta << 16 (bit p = orbital p).  A Pauli group with mask x
// maps the row of occupation n to occupation n ^ u, u = beta^-1 x.
struct SecDev {
  int32_t D;
  int no, na, nb;
  uint32_t cb;
  const uint32_t* occ;      // row -> occupation
  const uint32_t* kq;       // row -> qubit basis state
  const uint32_t* rank_a;   // alpha string -> rank (2^no entries)
  const uint32_t* rank_b;
};

// Row of occupation n ^ u, false when it leaves the sector.
__device__ __forceinline__ bool sec_row(const SecDev& s, uint32_t n, uint32_t u, uint32_t* r) {
  const uint32_t m = n ^ u, a = m & 0xFFFFu, b = m >> 16;
  if (__popc(a) != s.na || __popc(b) != s.nb) return false;
  *r = s.rank_a[a] * s.cb + s.rank_b[b];
  return true;
}

// Nonzero-octet masks (bit o of word o >> 5: octet o = amplitudes 8o..8o+7).
__device__ __forceinline__ uint32_t octet_bit(const uint32_t* mask, uint32_t b) {
  return (mask[b >> 8] >> ((b >> 3) & 31u)) & 1u;
}
__device__ __forceinline__ void octet_set(uint32_t* mask, uint32_t b) {
  atomicOr(mask + (b >> 8), 1u << ((b >> 3) & 31u));
}

// mask = exact nonzero-octet mask of psi (of psi or psi2 when psi2 is set),
// 2^(n-3) bits, n >= 8; resets *tile_counter when it is set; with
// tile_flags (zeroed by the caller) also sets bit t for every tile t (octets
// o >> tile_shift == t) holding a nonzero amplitude.  Defined in
// apply_tiled.cu.
int octet_mask(int precision, const void* psi, const void* psi2, int n, uint32_t* mask,
               unsigned int* tile_counter, int sm_count, cudaStream_t st, uint32_t* tile_flags = nullptr,
               int tile_shift = 0);

// The live octets of a state (those the nonzero-octet mask marks), listed in
// index order (the live-octet pool-gradient kernel), with the per-block
// counts of the listing pass and the length.
//
// The tiled form adds the nonzero amplitudes of a state in index order
// (aidx: index, aval: value; at most acap of them are stored, alen = their
// number, which may exceed acap), their per-block counts and offsets, and
// the first amplitude entry of every tile: toff[u] .. toff[u+1] are the
// nonzero amplitudes of tile u.
struct LiveOctets {
  uint32_t* list = nullptr;     // 2^(n-3) entries
  uint32_t* counts = nullptr;   // one per listing block
  uint32_t* len = nullptr;      // one entry
  uint32_t* toff = nullptr;     // 2^(n-LB) + 1 entries
  uint32_t* aidx = nullptr;     // acap entries
  void* aval = nullptr;         // acap complex amplitudes of the problem's precision
  uint32_t acap = 0;
  uint32_t* alen = nullptr;     // one entry
  uint32_t* acounts = nullptr;  // one per block of 256 amplitude words (32 amplitudes each), + 1
  unsigned long long* amax = nullptr;   // bits of max(|Re|, |Im|) over the listed amplitudes, as a double
  // scatter kernel with several blocks per output tile (few tiles): the
  // tiles' 64-bit fixed-point accumulators in global memory and a per-tile
  // count of finished blocks, both zero between calls (gtiles tiles; 0: none)
  unsigned long long* gacc = nullptr;
  unsigned int* tdone = nullptr;
  uint32_t gtiles = 0;
};

// Lists the live octets of `mask` (2^(n-3) bits, n >= 8) into lv.list and
// lv.len.  Defined in kernels.cu.
int live_octets(const uint32_t* mask, int n, const LiveOctets& lv, cudaStream_t st);

// H psi (+ the energy epilogue when partials is set) by the tiled kernels;
// t.n_pieces must be > 0.  States whose nonzero amplitudes are at most the
// fraction GOCP_SPARSE_FRAC (default 0.125, at most 0.25) of all take the
// scatter kernel of apply_sparse.cu, the others the staged kernel; the
// choice is made on the device from the count.  Defined in apply_tiled.cu.
int tiled_apply_h(const DevTables& t, const LiveOctets& lv, int precision, int sm_count, const void* psi,
                  void* hpsi, double identity, double* partials, unsigned int* counter,
                  unsigned int* tile_counter, double* scal, int32_t* err, cudaStream_t st);

// Pieces the scatter kernel takes (two bytes of shared memory each); a
// problem with more keeps every state on the staged kernel.
constexpr int kSpMaxPieces = 4096;

// Arguments of the scatter kernel (apply_sparse.cu); see sparse_apply_h.
template <typename R>
struct SparseArgs {
  const uint8_t* blob;
  const TiledPiece* piece;
  const uint32_t* porder;       // pieces by descending blob size (work units are numbered in this order)
  int n_pieces, n;
  const C_t<R>* psi;
  C_t<R>* out;
  const uint32_t* mask;
  const uint32_t* aidx;
  const C_t<R>* aval;
  const uint32_t* alen;
  const uint32_t* toff;
  const unsigned long long* amax;   // max(|Re|, |Im|) of the listed amplitudes (double bits)
  double hbound;                // DevTables::hbound
  double dmax;                  // DevTables::dmax
  const uint8_t* wfix;          // DevTables::twfix (complex128)
  double wscale;                // DevTables::twscale (complex128)
  uint32_t parts;               // blocks per output tile (>= 1; > 1 needs gacc, tdone)
  unsigned long long* gacc;     // LiveOctets::gacc
  unsigned int* tdone;          // LiveOctets::tdone
  uint32_t max_amps;            // the kernel runs only when *alen <= max_amps (<= acap)
  uint32_t n_offdiag;           // off-diagonal groups (LUT and term-list): products per accumulator word
  const uint32_t* dz;
  const R* dw;
  int nd, nd_mid;
  double identity;
  double* partials;
  unsigned int* counter;
  unsigned int* tile_counter;   // reset by octet_mask
  double* scal;
};

// Lists the amplitudes nonzero in psi or lam into cl (index order, the first
// cl.cap of them), writes cl.amask, and sets the ring so that a step whose
// previous slot is `slot` starts from the whole list: base(slot) = count,
// count(slot) = 0, and the first step's count(first) = 0; mask
// must mark every octet where psi or lam is nonzero.  Defined in
// apply_sparse.cu.
int chain_list(int precision, const void* psi, const void* lam, const uint32_t* mask, int n, const ChainList& cl,
               uint32_t* counts, int slot, int first, cudaStream_t st);

// Lists the nonzero amplitudes of psi into lv.aidx / lv.aval (index order,
// the first lv.acap of them) and their number into lv.alen; mask must mark
// every octet of psi holding a nonzero amplitude (extra set bits only cost
// time).  Defined in apply_sparse.cu.
int amp_list(int precision, const void* psi, const uint32_t* mask, int n, const LiveOctets& lv, cudaStream_t st);

// Lists the nonzero amplitudes of a.psi (whose exact octet mask is a.mask)
// into lv, their tile offsets, and launches the scatter H psi kernel, a
// no-op on the device when there are more than a.max_amps; a.aidx, a.aval,
// a.alen and a.toff are taken from lv.  Defined in apply_sparse.cu.
template <typename R>
int sparse_apply_h(SparseArgs<R> a, const LiveOctets& lv, int sm_count, cudaStream_t st);

// Accessors of a problem's device state for the sector-layout launchers
// (defined in kernels.cu).
struct Problem;
const DevTables& dev_tables(Problem& p);
double* coefs_ptr(Problem& p);
double* scratch_ptr(Problem& p, size_t* doubles);
unsigned int* counters_ptr(Problem& p);
int pool_finish(Problem& p, const double* part, int nbx, double* d_grads, cudaStream_t st);
int ensure_stage(Problem& p, int n_ops);
double* scalars_ptr(Problem& p);
int32_t* err_ptr(Problem& p);
int dev_norm(Problem& p, const void* psi, cudaStream_t st);

}  // namespace gocp
