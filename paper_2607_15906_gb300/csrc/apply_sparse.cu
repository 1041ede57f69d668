// H psi (Eq. 3) with the energy epilogue (Eq. 1) for states whose nonzero
// amplitudes fill few octets, by scattering from the live source octets.
//
// The staged kernel (apply_tiled.cu) gives every thread an output octet and
// walks the groups of a piece; a group is skipped only where the source
// octet is zero, so in a state confined to a particle-number sector (8.9 %
// of octets live at 24 qubits) most lanes of a warp idle while a few work.
// This kernel turns the loop around.  A block owns an output tile t of 2^LB
// amplitudes and accumulates it in shared memory; for each piece (groups of
// one x >> LB, source tile u = t ^ (x >> LB)) its warps take the live octets
// l of u, 32 at a time (one per lane, from the index-ordered live list), load
// each lane's 8 source amplitudes once, and walk the piece's groups together:
// group g sends source octet l to output octet l ^ s_g (s_g = (x >> 3) within
// the tile), output member i taking source member i ^ (x & 7) with
// D_g(k) computed exactly as in the staged kernel (LUT entries, Walsh
// buckets, paired or term-by-term).  Every product that is nonzero (D and
// the source amplitude both nonzero) is added to the tile's accumulator with
// a shared-memory atomic; a product with a zero factor is exactly zero and
// is left out.  After the last piece the block adds the diagonal group and
// the identity on the live octets of its own tile, the energy partials, and
// streams the whole tile (zeros included) to H psi.
//
// The order in which products reach an accumulator element is not fixed, so
// the result may differ from run to run in the last bits of a sum (and from
// the staged kernel's fixed order); every term is the same.
//
// The kernel is launched with the staged one; each returns at once unless
// the live count selects it, so the choice needs no host round trip.
#include <algorithm>
#include <mutex>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace gocp {

namespace {

constexpr int kSpThreads = 512;

// The tile's accumulator is component-major: component j (2i: real part,
// 2i + 1: imaginary part of member i) of octet o at j * kOct + o, so that
// the epilogue's reads are consecutive and a warp's atomics on one component
// spread over the banks by octet.
template <typename R>
__device__ __forceinline__ void acc_add(R* acc, uint32_t at, R re, R im, uint32_t koct) {
  atomicAdd(acc + at, re);
  atomicAdd(acc + at + koct, im);
}

// The group arithmetic is indexed by the lane's source member m: output
// member i = m ^ xl (xl = x & 7 of the run) takes source member m.  Every
// sign and LUT code is linear in the index over GF(2), so evaluating them at
// k0x = k0 | xl (k0 = first index of the output octet) gives at member m the
// value of output index k0 + (m ^ xl); xl then enters only the accumulator
// address, and one code path serves every xl.

// LUT groups of one run: l = the lane's source octet within its tile, src
// its amplitudes, nz its nonzero members; kb = first index of the output
// tile.  Every member looks its entry up: members that differ only in bits
// outside the group's flip class have the same code (tiled_flip_class), so
// those lookups read one word.
template <typename R, uint32_t kOct>
__device__ __forceinline__ void sp_lut(const HLut<R>* __restrict__ ls, int cn, uint32_t xl, uint32_t kb, uint32_t l,
                                       const C_t<R> (&src)[kAmpsH], uint32_t nz, R* acc) {
  for (int g = 0; g < cn; ++g) {
    const HLut<R>& L = ls[g];
    const uint4 h0 = *reinterpret_cast<const uint4*>(&L.x);     // x, z0, v0, v1
    const uint4 h1 = *reinterpret_cast<const uint4*>(&L.v2);    // v2, reg, pad0, pad1
    const uint32_t ol = l ^ h1.w, k0x = kb | (ol << 3) | xl, reg = h1.y;
    const uint32_t code0 = (uint32_t)(__popc(k0x & h0.z) & 1) | ((uint32_t)(__popc(k0x & h0.w) & 1) << 1) |
                           ((uint32_t)(__popc(k0x & h1.x) & 1) << 2) | ((uint32_t)(__popc(k0x & h0.y) & 1) << 3);
#pragma unroll
    for (int m = 0; m < kAmpsH; ++m) {
      const R v = L.lut16[code0 ^ ((reg >> (4 * m)) & 0xFu)];
      if (v != R(0) && ((nz >> m) & 1u))
        acc_add<R>(acc, ((2u * ((uint32_t)m ^ xl)) * kOct) + ol, v * src[m].x, v * src[m].y, kOct);
    }
  }
}

// Term-list groups of one run: paired, Walsh-bucketed or term by term.
template <typename R, uint32_t kOct>
__device__ __forceinline__ void sp_terms(const TiledGroup* __restrict__ gs, int cn, uint32_t xl,
                                         const uint32_t* __restrict__ zs, const R* __restrict__ ws, uint32_t kb,
                                         uint32_t l, const C_t<R> (&src)[kAmpsH], uint32_t nz, R* acc) {
  for (int g = 0; g < cn; ++g) {
    const TiledGroup& G = gs[g];
    const uint32_t ol = l ^ G.pad, k0x = kb | (ol << 3) | xl;
    if (G.delta || G.bk != ~0ull) {
      uint32_t live = 0xFFu;
      if (G.delta) {
        // paired: D = (1 + sigma (-1)^popc(k & delta)) E, the factor 0 or 2
        const uint32_t f = octet_signs(k0x, G.delta);
        live = G.neg ? f : (~f & 0xFFu);
      }
      live &= nz;
      if (!live) continue;
      // bucket m': the terms with z & 7 == m'; D at member m is
      // sum_m' B_m' (-1)^popc(m & m') (a Walsh transform)
      R b[kAmpsH];
      int t = (int)G.tb;
#pragma unroll
      for (int m = 0; m < kAmpsH; ++m) {
        b[m] = R(0);
        const int cnt = (int)((G.bk >> (8 * m)) & 0xFFu);
        for (int c = 0; c < cnt; ++c, ++t) b[m] += (__popc(k0x & zs[t]) & 1) ? -ws[t] : ws[t];
      }
#pragma unroll
      for (int hb = 1; hb < kAmpsH; hb <<= 1)
#pragma unroll
        for (int q = 0; q < kAmpsH; ++q)
          if (!(q & hb)) {
            const R u = b[q], v = b[q | hb];
            b[q] = u + v;
            b[q | hb] = u - v;
          }
      const R f2 = G.delta ? R(2) : R(1);
#pragma unroll
      for (int m = 0; m < kAmpsH; ++m) {
        const R d = f2 * b[m];
        if (((live >> m) & 1u) && d != R(0))
          acc_add<R>(acc, ((2u * ((uint32_t)m ^ xl)) * kOct) + ol, d * src[m].x, d * src[m].y, kOct);
      }
      continue;
    }
    if (!nz) continue;
    R gr[kAmpsH], gi[kAmpsH], cr[kAmpsH], ci[kAmpsH];
#pragma unroll
    for (int m = 0; m < kAmpsH; ++m) gr[m] = gi[m] = cr[m] = ci[m] = R(0);
    sum_terms8<R>(zs, ws, (int)G.tb, (int)G.tm, k0x, gr, cr, false);
    if (G.te > G.tm) sum_terms8<R>(zs, ws, (int)G.tm, (int)G.te, k0x, gi, ci, false);
#pragma unroll
    for (int m = 0; m < kAmpsH; ++m)
      if (((nz >> m) & 1u) && (gr[m] != R(0) || gi[m] != R(0))) {
        const C_t<R> p = src[m];
        acc_add<R>(acc, ((2u * ((uint32_t)m ^ xl)) * kOct) + ol, gr[m] * p.x - gi[m] * p.y, gr[m] * p.y + gi[m] * p.x,
                   kOct);
      }
  }
}

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

// off[u] = first entry of the index-ordered live list in tile u (octets
// o >> shift == u), u = 0 .. ntiles; off[ntiles] = the list's length.
__global__ void __launch_bounds__(256)
k_tile_offsets(const uint32_t* __restrict__ list, const uint32_t* __restrict__ len, uint32_t ntiles, int shift,
               uint32_t* off) {
  const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u > ntiles) return;
  uint32_t lo = 0, hi = *len;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((list[mid] >> shift) < u) lo = mid + 1;
    else hi = mid;
  }
  off[u] = lo;
}

template <typename R>
__global__ void __launch_bounds__(kSpThreads, sizeof(R) == 4 ? 2 : 1) k_apply_h_sparse(const SparseArgs<R> a) {
  constexpr int LB = TiledBits<R>::LB;
  constexpr uint32_t kOct = 1u << (LB - 3);   // octets per tile
  if (*a.len > a.max_live) return;            // the staged kernel takes this state
  extern __shared__ __align__(16) uint8_t sp_raw[];
  R* acc = reinterpret_cast<R*>(sp_raw);      // 16 components x kOct octets
  __shared__ uint32_t s_tile, s_unext, s_maxch;
  __shared__ uint8_t s_nch[kSpMaxPieces];
  __shared__ double tot[2];
  const uint32_t ntiles = 1u << (a.n - LB);
  const int lane = threadIdx.x & 31;
  for (uint32_t j = threadIdx.x; j < kOct * 16u; j += kSpThreads) acc[j] = R(0);
  const R idr = (R)a.identity;
  // this thread's |psi|^2 and <psi|H - identity|psi> partials (in shared
  // memory: touched once per tile)
  __shared__ double2 s_v[kSpThreads];
  s_v[threadIdx.x] = make_double2(0.0, 0.0);
  for (;;) {
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(a.tile_counter, 1u);
      s_unext = 0u;
      s_maxch = 0u;
    }
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= ntiles) break;
    const uint32_t kb = t << LB;
    // scatter.  Work units are (chunk c, piece p): the live octets
    // 32c .. 32c + 31 of p's source tile u = t ^ (x >> LB) against p's groups.
    // The units are handed out chunk-major from a block counter, so that the
    // last units of the tile are small; s_nch[p] = p's chunk count.
    for (int p = (int)threadIdx.x; p < a.n_pieces; p += kSpThreads) {
      const TiledPiece pc = a.piece[p];
      const uint32_t u = t ^ pc.xhi;
      const uint32_t nch = pc.bytes ? (a.toff[u + 1] - a.toff[u] + 31u) >> 5 : 0u;
      s_nch[p] = (uint8_t)nch;
      if (nch) atomicMax(&s_maxch, nch);
    }
    __syncthreads();
    const uint32_t P = (uint32_t)a.n_pieces, n_units = s_maxch * P;
    for (;;) {
      uint32_t j = 0;
      if (lane == 0) j = atomicAdd(&s_unext, 1u);
      j = __shfl_sync(0xffffffffu, j, 0);
      if (j >= n_units) break;
      const uint32_t c = j / P, p = j - c * P;
      if (c >= s_nch[p]) continue;
      const TiledPiece pc = a.piece[p];
      const uint32_t u = t ^ pc.xhi;
      const uint32_t l0 = a.toff[u], l1 = a.toff[u + 1];
      const uint8_t* bl = a.blob + pc.off;
      const TiledHead* hd = reinterpret_cast<const TiledHead*>(bl);
      const HLut<R>* ls = reinterpret_cast<const HLut<R>*>(bl + sizeof(TiledHead));
      const TiledGroup* gs = reinterpret_cast<const TiledGroup*>(bl + sizeof(TiledHead) + hd->n_lut * sizeof(HLut<R>));
      const uint32_t* zs = reinterpret_cast<const uint32_t*>(bl + hd->z_off);
      const R* ws = reinterpret_cast<const R*>(bl + hd->w_off);
      const int nr = (int)hd->n_runs;
      const uint32_t li = l0 + 32u * c + (uint32_t)lane;
      const bool valid = li < l1;
      const uint32_t so = a.list[valid ? li : l0];
      C_t<R> src[kAmpsH];
      load_octet<R>(a.psi, so, src);
      uint32_t nz = 0;
#pragma unroll
      for (int m = 0; m < kAmpsH; ++m) nz |= (uint32_t)(src[m].x != R(0) || src[m].y != R(0)) << m;
      if (!valid) nz = 0;
      const uint32_t l = so & (kOct - 1u);
      for (int r = 0; r < nr; ++r) {
        const uint32_t rd = hd->run[r];
        const int g0 = (int)(rd & 0xFFFu), cn = (int)((rd >> 12) & 0xFFFu) - g0;
        const uint32_t sel = rd >> 24, xl = sel & 7u;
        if (sel < 64) sp_lut<R, kOct>(ls + g0, cn, xl, kb, l, src, nz, acc);
        else sp_terms<R, kOct>(gs + g0, cn, xl, zs, ws, kb, l, src, nz, acc);
      }
    }
    __syncthreads();
    // epilogue: diagonal, identity and energy on the live own octets; the
    // whole tile out; the accumulator cleared for the next tile
    for (uint32_t o = threadIdx.x; o < kOct; o += kSpThreads) {
      C_t<R> res[kAmpsH];
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) {
        R* e = acc + (2u * i) * kOct + o;
        res[i] = cmake<R>(e[0], e[kOct]);
        e[0] = R(0);
        e[kOct] = R(0);
      }
      const uint32_t go = (t << (LB - 3)) | o, k0 = go << 3;
      if ((a.mask[go >> 5] >> (go & 31u)) & 1u) {
        R dr[kAmpsH], dc[kAmpsH], di[kAmpsH], dd[kAmpsH];
#pragma unroll
        for (int i = 0; i < kAmpsH; ++i) dr[i] = dc[i] = di[i] = dd[i] = R(0);
        sum_terms8<R>(a.dz, a.dw, 0, a.nd_mid, k0, dr, dc, true);
        sum_terms8<R>(a.dz, a.dw, a.nd_mid, a.nd, k0, di, dd, false);
        C_t<R> own[kAmpsH];
        load_octet<R>(a.psi, go, own);
        double2 v = s_v[threadIdx.x];
#pragma unroll
        for (int i = 0; i < kAmpsH; ++i) {
          const C_t<R> q = own[i];
          const double pp = (double)q.x * q.x + (double)q.y * q.y;
          v.x += pp;
          v.y += (double)q.x * res[i].x + (double)q.y * res[i].y + ((double)dr[i] - (double)dc[i]) * pp;
          const R d0 = dr[i] - dc[i] + idr;
          res[i] = cmake<R>(res[i].x + d0 * q.x - di[i] * q.y, res[i].y + d0 * q.y + di[i] * q.x);
        }
        s_v[threadIdx.x] = v;
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
  if (a.partials && block_grid_sum<2, kSpThreads>(v, a.partials, a.counter, gridDim.x, blockIdx.x, a.scal + 1, tot)) {
    if (threadIdx.x == 0) a.scal[0] = a.identity + tot[1] / tot[0];
  }
}

template <typename R>
constexpr uint32_t sparse_smem() {
  return (1u << (TiledBits<R>::LB - 3)) * 16u * (uint32_t)sizeof(R);
}

}  // namespace

template <typename R>
int sparse_apply_h(SparseArgs<R> a, const LiveOctets& lv, int sm_count, cudaStream_t st) {
  constexpr int LB = TiledBits<R>::LB;
  if (a.n < LB || !lv.toff || !lv.list || !lv.len) return fail(GOCP_EINVAL, "scatter H psi needs the live list");
  a.list = lv.list;
  a.len = lv.len;
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
  const uint32_t ntiles = 1u << (a.n - LB);
  k_tile_offsets<<<(ntiles + 256u) / 256u, 256, 0, st>>>(lv.list, lv.len, ntiles, LB - 3, lv.toff);
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)std::max(sm_count, 1) * 2u);
  k_apply_h_sparse<R><<<grid, kSpThreads, sparse_smem<R>(), st>>>(a);
  count_launches(2);
  return cuda_status(cudaGetLastError(), "k_apply_h_sparse");
}

template int sparse_apply_h<float>(SparseArgs<float>, const LiveOctets&, int, cudaStream_t);
template int sparse_apply_h<double>(SparseArgs<double>, const LiveOctets&, int, cudaStream_t);

}  // namespace gocp
