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
  // diagonal group (x = 0) without the identity: [0, nd_mid) real, [nd_mid, nd) imaginary
  int nd = 0, nd_mid = 0;
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
};

}  // namespace gocp
