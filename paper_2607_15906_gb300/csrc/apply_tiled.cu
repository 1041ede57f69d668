// H psi (Eq. 3) with the energy epilogue (Eq. 1), by shared-memory tiles.
//
// A block owns output tiles of 2^LB amplitudes (64 KiB), one octet k0..k0+7
// per thread.  A group with mask x sends source tile (tile ^ (x >> LB)) to
// the output tile, so the groups are cut into pieces of equal x >> LB
// (TiledHead): per piece the block stages that source tile in shared memory
// with one TMA tensor copy per 256 rows of 128 bytes (128-byte swizzle, so
// that the octet reads of a warp hit 32 distinct banks) and the piece's
// descriptor blob with one bulk copy, both completing on one mbarrier.  Two
// stages alternate: while the block computes piece i, the copies of piece
// i + 1 are in flight.  The arithmetic per group is the one of the untiled
// kernel: LUT groups D(k) = lut16[code(k)], term-list groups by Walsh
// buckets or term by term, the x & 7 permutation resolved at compile time.
// The pieces with x >> LB = 0 come last, so that the own tile is staged when
// the diagonal group and the energy terms are added.
//
// A pre-pass (k_octet_mask) marks the octets of psi that hold a nonzero
// amplitude; each piece's copy brings the source tile's slice of that mask,
// and a group skips a source octet that is entirely zero (its contribution is
// exactly zero).  States confined to a particle-number sector, as the ADAPT
// states are, leave most octets zero; a dense state skips nothing.
//
// Every staging wait on an mbarrier gives up after a limit of %globaltimer
// (2 s, or GOCP_STAGE_WAIT_NS nanoseconds from the environment): the block
// then records bit 1 in the error flags, waits -- always with the full 2 s
// limit -- for its own copies in flight, and leaves the tile loop; results
// are then undefined and gocp_device_errors reports the flag.
#include <cuda.h>

#include <cmath>
#include <cstdlib>

#include <mutex>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace gocp {

namespace {

constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s
constexpr int32_t kErrStageTimeout = 2;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity to complete; false after
// limit_ns of %globaltimer.  A limit of 0 gives up without looking (the
// abort path on every call, for a test).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (limit_ns == 0) return false;
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 32; ++i)
      if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// Rows [row, row + box) of the tensor map into shared memory; the lines are
// marked to stay in L2 (evict_last policy), since every tile of the state is
// read again by other pieces while the output streams past.
__device__ __forceinline__ void tma_rows(uint32_t dst, const CUtensorMap* map, int row, uint32_t bar,
                                         uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(bar), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// The octet at byte offset `off` (tiled_swz) of a staged tile.
template <typename R>
__device__ __forceinline__ void tile_octet(const uint8_t* tile, uint32_t off, C_t<R> (&v)[kAmpsH]) {
  if (sizeof(R) == 4) {
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const float4 f = *reinterpret_cast<const float4*>(tile + (off ^ (q << 4)));
      v[2 * q] = cmake<R>((R)f.x, (R)f.y);
      v[2 * q + 1] = cmake<R>((R)f.z, (R)f.w);
    }
  } else {
#pragma unroll
    for (uint32_t q = 0; q < 8; ++q) {
      const double2 f = *reinterpret_cast<const double2*>(tile + (off ^ (q << 4)));
      v[q] = cmake<R>((R)f.x, (R)f.y);
    }
  }
}

// Whether source octet so of the staged tile holds a nonzero amplitude (mk:
// the tile's slice of the nonzero-octet mask).  Within a warp so >> 5 is
// uniform, so a zero 32-octet block skips a group for the whole warp; a
// group's product with zero amplitudes is zero, so skipping changes nothing.
__device__ __forceinline__ bool octet_live(const uint32_t* mk, uint32_t so) {
  return (mk[so >> 5] >> (so & 31u)) & 1u;
}

// LUT groups of one run: x & 7 == XL and flip class F (tiled_flip_class);
// k0 = first global index of the thread's output octet, o its octet in the
// tile and ao = tiled_swz(o).  Member i of the octet takes the LUT entry of
// member i & F, so only the 2^popc(F) members i == i & F are looked up.
template <typename R, int XL, int F>
__device__ __forceinline__ void tiled_lut(const HLut<R>* ls, int cn, uint32_t k0, uint32_t o, uint32_t ao,
                                          const uint8_t* tile, const uint32_t* mk, C_t<R> (&acc)[kAmpsH]) {
  for (int g = 0; g < cn; ++g) {
    const HLut<R>& L = ls[g];
    if (!octet_live(mk, o ^ L.pad1)) continue;
    const uint32_t os = ao ^ L.pad0, reg = L.reg;
    const uint32_t code0 = (uint32_t)(__popc(k0 & L.v0) & 1) | ((uint32_t)(__popc(k0 & L.v1) & 1) << 1) |
                           ((uint32_t)(__popc(k0 & L.v2) & 1) << 2) | ((uint32_t)(__popc(k0 & L.z0) & 1) << 3);
    R val[kAmpsH];
    bool any = false;
#pragma unroll
    for (int i = 0; i < kAmpsH; ++i)
      if ((i & F) == i) {
        val[i] = L.lut16[code0 ^ ((reg >> (4 * i)) & 0xFu)];
        any |= val[i] != R(0);
      }
#pragma unroll
    for (int i = 0; i < kAmpsH; ++i)
      if ((i & F) != i) val[i] = val[i & F];
    if (!any) continue;   // no output of this octet couples to the group
    C_t<R> src[kAmpsH];
    tile_octet<R>(tile, os, src);
#pragma unroll
    for (int i = 0; i < kAmpsH; ++i) {
      acc[i].x += val[i] * src[i ^ XL].x;
      acc[i].y += val[i] * src[i ^ XL].y;
    }
  }
}

// Term-list groups of one x & 7 run.
template <typename R, int XL>
__device__ __forceinline__ void tiled_terms(const TiledGroup* gs, int cn, const uint32_t* zs, const R* ws,
                                            uint32_t k0, uint32_t o, uint32_t ao, const uint8_t* tile,
                                            const uint32_t* mk, C_t<R> (&acc)[kAmpsH]) {
  for (int g = 0; g < cn; ++g) {
    const TiledGroup& G = gs[g];
    if (!octet_live(mk, o ^ G.pad)) continue;
    const uint32_t os = ao ^ G.xa;
    if (G.delta) {
      // paired: D = (1 + sigma (-1)^popc(k & delta)) E, the factor 0 or 2
      const uint32_t f = octet_signs(k0, G.delta);
      const uint32_t live = G.neg ? f : (~f & 0xFFu);
      if (!live) continue;
      R b[kAmpsH];
      int t = (int)G.tb;
#pragma unroll
      for (int m = 0; m < kAmpsH; ++m) {
        b[m] = R(0);
        const int cnt = (int)((G.bk >> (8 * m)) & 0xFFu);
        for (int c = 0; c < cnt; ++c, ++t) b[m] += (__popc(k0 & zs[t]) & 1) ? -ws[t] : ws[t];
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
      C_t<R> src[kAmpsH];
      tile_octet<R>(tile, os, src);
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) {
        const R d = ((live >> i) & 1u) ? R(2) * b[i] : R(0);
        acc[i].x += d * src[i ^ XL].x;
        acc[i].y += d * src[i ^ XL].y;
      }
      continue;
    }
    if (G.bk != ~0ull) {
      // bucket m: the terms with z & 7 == m, summed with the signs of k0;
      // D(k0 + i) = sum_m B_m (-1)^popc(i & m)
      R b[kAmpsH];
      int t = (int)G.tb;
#pragma unroll
      for (int m = 0; m < kAmpsH; ++m) {
        b[m] = R(0);
        const int cnt = (int)((G.bk >> (8 * m)) & 0xFFu);
        for (int c = 0; c < cnt; ++c, ++t) b[m] += (__popc(k0 & zs[t]) & 1) ? -ws[t] : ws[t];
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
      C_t<R> src[kAmpsH];
      tile_octet<R>(tile, os, src);
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
    sum_terms8<R>(zs, ws, (int)G.tb, (int)G.tm, k0, gr, cr, false);
    if (G.te > G.tm) sum_terms8<R>(zs, ws, (int)G.tm, (int)G.te, k0, gi, ci, false);
    C_t<R> src[kAmpsH];
    tile_octet<R>(tile, os, src);
#pragma unroll
    for (int i = 0; i < kAmpsH; ++i) {
      const C_t<R> p = src[i ^ XL];
      acc[i].x += gr[i] * p.x - gi[i] * p.y;
      acc[i].y += gr[i] * p.y + gi[i] * p.x;
    }
  }
}

// mask bit o = octet o of psi (or of psi2, when set) holds a nonzero
// amplitude (-0 counts as zero); one ballot word per warp of 32 octets.
template <typename R>
__device__ __forceinline__ bool octet_nonzero(const C_t<R>* psi, uint32_t o) {
  bool nz = false;
  if (sizeof(R) == 4) {
    const float4* p = reinterpret_cast<const float4*>(psi) + 4u * o;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 f = p[q];
      nz |= (f.x != 0.f) | (f.y != 0.f) | (f.z != 0.f) | (f.w != 0.f);
    }
  } else {
    const double2* p = reinterpret_cast<const double2*>(psi) + 8u * o;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double2 f = p[q];
      nz |= (f.x != 0.0) | (f.y != 0.0);
    }
  }
  return nz;
}

// With tile_flags set (zeroed before), bit t of it is set when tile t (the
// octets o with o >> tile_shift == t) holds a nonzero amplitude.
template <typename R>
__global__ void __launch_bounds__(256) k_octet_mask(const C_t<R>* __restrict__ psi, const C_t<R>* __restrict__ psi2,
                                                    uint32_t n_octets, uint32_t* __restrict__ mask,
                                                    unsigned int* tile_counter, uint32_t* tile_flags,
                                                    int tile_shift) {
  if (tile_counter && blockIdx.x == 0 && threadIdx.x == 0) *tile_counter = 0u;   // for the H psi kernel that follows
  for (uint32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < n_octets; o += gridDim.x * blockDim.x) {
    bool nz = octet_nonzero<R>(psi, o);
    if (psi2) nz |= octet_nonzero<R>(psi2, o);
    const uint32_t w = __ballot_sync(0xffffffffu, nz);
    if ((threadIdx.x & 31u) == 0) {
      mask[o >> 5] = w;
      if (w && tile_flags) {
        const uint32_t t = o >> tile_shift;
        atomicOr(tile_flags + (t >> 5), 1u << (t & 31u));
      }
    }
  }
}

template <typename R>
struct TiledArgs {
  const uint8_t* blob;
  const TiledPiece* piece;
  const uint32_t* mask;   // nonzero-octet mask of the source state
  unsigned int* tile_counter;   // next output tile to claim (zeroed by k_octet_mask)
  const uint32_t* tile_flags;   // bit t: source tile t holds a nonzero amplitude (k_octet_mask)
  int n_pieces;
  int n;
  const uint32_t* dz;   // diagonal group: [0, nd_mid) real, [nd_mid, nd) imaginary
  const R* dw;
  int nd, nd_mid;
  C_t<R>* out;
  double identity;
  double* partials;     // null: no energy
  unsigned int* counter;
  double* scal;
  int32_t* err;
  // set: the kernel returns at once when *gate <= gate_max (the scatter
  // kernel of apply_sparse.cu takes the state)
  const uint32_t* gate;
  uint32_t gate_max;
  uint64_t wait_ns;     // limit of a staging wait (stage_wait_ns)
};

template <typename R>
__host__ __device__ constexpr uint32_t tile_bytes() {
  return (1u << TiledBits<R>::LB) * (uint32_t)sizeof(C_t<R>);
}

template <typename R>
__host__ __device__ constexpr int tiled_threads() {
  return 1 << (TiledBits<R>::LB - 3);
}

// bytes of the nonzero-octet mask of one tile (one bit per octet)
template <typename R>
__host__ __device__ constexpr uint32_t tile_mask_bytes() {
  return (1u << (TiledBits<R>::LB - 3)) / 8u;
}

// pipeline stages: copies of up to stages - 1 pieces in flight (complex64
// may use more with smaller tiles; complex128 tiles take 64 KiB each)
#ifndef GOCP_TILED_STAGES_C64
#define GOCP_TILED_STAGES_C64 3
#endif
template <typename R>
__host__ __device__ constexpr int tiled_stages() {
  return sizeof(R) == 4 ? GOCP_TILED_STAGES_C64 : 3;
}

template <typename R>
__host__ __device__ constexpr size_t tiled_smem() {
  return 1024 + tiled_stages<R>() * ((size_t)tile_bytes<R>() + (size_t)kTiledBlobBytes + (size_t)tile_mask_bytes<R>());
}

// resident blocks per SM the register budget must allow
#ifndef GOCP_TILED_MINB_C64
#define GOCP_TILED_MINB_C64 1
#endif

template <typename R>
__global__ void __launch_bounds__(tiled_threads<R>(), sizeof(R) == 4 ? GOCP_TILED_MINB_C64 : 1)
    k_apply_h_tiled(const __grid_constant__ CUtensorMap tmap, const TiledArgs<R> a) {
  constexpr int LB = TiledBits<R>::LB;
  constexpr int NT = tiled_threads<R>();
  constexpr uint32_t kTile = tile_bytes<R>();
  constexpr uint32_t kRows = kTile / 128u;
  constexpr uint32_t kBox = kRows < 256u ? kRows : 256u;
  constexpr uint32_t kMask = tile_mask_bytes<R>();
  static_assert(kMask % 16u == 0, "mask slices are whole 16-byte units");
  if (a.gate && *a.gate <= a.gate_max) return;   // the same answer for every thread
  constexpr int S = tiled_stages<R>();
  constexpr uint32_t kWarps = NT / 32;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[S], bar_empty[S];
  __shared__ volatile int s_abort;
  __shared__ double tot[2];
  // stage st: tile at base + st kTile, blob at base + S kTile + st kBlob,
  // mask slice at base + S (kTile + kBlob) + st kMask
  uint8_t* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const uint32_t base_s = smem_addr(base), full_s = smem_addr(&bar_full[0]), empty_s = smem_addr(&bar_empty[0]);
  constexpr uint32_t kBlobOff = S * kTile, kMaskOff = S * (kTile + kTiledBlobBytes);

  // Items are (tile, piece) pairs.  Output tiles are claimed one at a time
  // from a global counter when their first piece is issued (tiles differ in
  // cost when zero octets are skipped), and the tile of each staged item is
  // passed to the consumers in s_tile; kNoTile ends the sweep.
  constexpr uint32_t kNoTile = 0xFFFFFFFFu;
  const uint32_t ntiles = 1u << (a.n - LB);
  __shared__ uint32_t s_tile[S], s_piece[S];
  // per-thread energy partials live in shared memory (touched once per tile)
  __shared__ double2 s_v[NT];
  s_v[threadIdx.x] = make_double2(0.0, 0.0);

  if (threadIdx.x == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(full_s + 8u * q, 1);
      mbar_init(empty_s + 8u * q, kWarps);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // producer state, thread 0 only, kept in shared memory (not in every
  // thread's registers): items issued, piece and tile of the next, done
  __shared__ uint32_t s_next, s_pnext, s_tnext, s_done;
  if (threadIdx.x == 0) s_next = s_pnext = s_tnext = s_done = 0u;
  // thread 0: issue item s_next into stage s_next % S, whose previous item
  // every warp has released.  A piece whose source tile holds no nonzero
  // amplitude adds nothing and is passed over (never the last piece of a
  // tile, which carries the diagonal and the output).  The stage's tile and
  // piece slots are written before the barrier arrive (release), so a
  // consumer that sees the phase complete (acquire) reads them.
  auto issue_next = [&]() {
    const uint32_t st = s_next % S;
    const uint32_t fb = full_s + 8u * st;
    uint32_t p = s_pnext, t = s_tnext;
    for (;;) {
      if (p == 0) t = atomicAdd(a.tile_counter, 1u);
      if (t >= ntiles) {
        s_tile[st] = kNoTile;
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fb) : "memory");
        s_done = 1u;
        ++s_next;
        return;
      }
      const uint32_t src = t ^ a.piece[p].xhi;
      if (p + 1u == (uint32_t)a.n_pieces || !a.tile_flags || ((a.tile_flags[src >> 5] >> (src & 31u)) & 1u)) break;
      ++p;
    }
    s_tile[st] = t;
    s_piece[st] = p;
    const TiledPiece pc = a.piece[p];
    const uint32_t src = t ^ pc.xhi;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(fb, kTile + pc.bytes + kMask);
    const uint64_t keep = policy_evict_last();
#pragma unroll
    for (uint32_t c = 0; c < kRows / kBox; ++c)
      tma_rows(base_s + st * kTile + c * kBox * 128u, &tmap, (int)(src * kRows + c * kBox), fb, keep);
    if (pc.bytes) bulk_copy(base_s + kBlobOff + st * kTiledBlobBytes, a.blob + pc.off, pc.bytes, fb);
    bulk_copy(base_s + kMaskOff + st * kMask, reinterpret_cast<const uint8_t*>(a.mask) + (size_t)src * kMask, kMask,
              fb);
    ++s_next;
    s_pnext = p + 1u == (uint32_t)a.n_pieces ? 0u : p + 1u;
    s_tnext = t;
  };
  // Item j (j >= S) may reuse its stage once every warp has released item
  // j - S: phase (j / S - 1) of that stage's empty barrier.
  if (threadIdx.x == 0)
    while (!s_done && s_next < (uint32_t)S) issue_next();

  const R idr = (R)a.identity;
  const uint32_t o = threadIdx.x, ao = tiled_swz<R>(o);
  C_t<R> acc[kAmpsH];
#pragma unroll
  for (int i = 0; i < kAmpsH; ++i) acc[i] = cmake<R>(0, 0);
  uint32_t it = 0, tile = 0, st = 0, ph = 0;
  for (;; ++it) {
    // every exit decision is warp-uniform, so that no lane leaves its warp
    // waiting in __syncwarp
    if (__shfl_sync(0xffffffffu, s_abort, 0)) break;
    if (threadIdx.x == 0) {
      // item it must be issued before anyone waits for it; later items go
      // out as soon as their stage is released
      bool ok = true;
      while (ok && !s_done && s_next <= it) {
        ok = mbar_wait(empty_s + 8u * (s_next % S), (s_next / S - 1u) & 1u, a.wait_ns);
        if (ok) issue_next();
      }
      while (ok && !s_done && mbar_try(empty_s + 8u * (s_next % S), (s_next / S - 1u) & 1u)) issue_next();
      if (!ok) s_abort = 1;
    }
    __syncwarp();
    if (!__all_sync(0xffffffffu, mbar_wait(full_s + 8u * st, ph, a.wait_ns))) {
      s_abort = 1;
      break;
    }
    tile = s_tile[st];
    if (tile == kNoTile) break;   // the same item, so the same answer, for every warp
    const int pc = (int)s_piece[st];
    {
      const uint32_t k0 = (tile << LB) + o * kAmpsH;
      const uint8_t* tl = base + st * kTile;
      const uint8_t* bl = base + kBlobOff + st * kTiledBlobBytes;
      const uint32_t* mk = reinterpret_cast<const uint32_t*>(base + kMaskOff + st * kMask);
      const TiledHead* hd = reinterpret_cast<const TiledHead*>(bl);
      const HLut<R>* ls = reinterpret_cast<const HLut<R>*>(bl + sizeof(TiledHead));
      const TiledGroup* gs = reinterpret_cast<const TiledGroup*>(bl + sizeof(TiledHead) + hd->n_lut * sizeof(HLut<R>));
      const uint32_t* zs = reinterpret_cast<const uint32_t*>(bl + hd->z_off);
      const R* ws = reinterpret_cast<const R*>(bl + hd->w_off);
      const int nr = (int)hd->n_runs;
      for (int r = 0; r < nr; ++r) {
        const uint32_t rd = hd->run[r];
        const int g0 = (int)(rd & 0xFFFu), cn = (int)((rd >> 12) & 0xFFFu) - g0;
        switch (rd >> 24) {
#define GOCP_LUT_CASE(SEL)                                                                    \
  case SEL:                                                                                   \
    tiled_lut<R, ((SEL) & 7), ((SEL) >> 3)>(ls + g0, cn, k0, o, ao, tl, mk, acc);             \
    break;
#define GOCP_LUT_CASES8(F8) GOCP_LUT_CASE(F8 + 0) GOCP_LUT_CASE(F8 + 1) GOCP_LUT_CASE(F8 + 2) \
  GOCP_LUT_CASE(F8 + 3) GOCP_LUT_CASE(F8 + 4) GOCP_LUT_CASE(F8 + 5) GOCP_LUT_CASE(F8 + 6) GOCP_LUT_CASE(F8 + 7)
          GOCP_LUT_CASES8(0) GOCP_LUT_CASES8(8) GOCP_LUT_CASES8(16) GOCP_LUT_CASES8(24)
          GOCP_LUT_CASES8(32) GOCP_LUT_CASES8(40) GOCP_LUT_CASES8(48) GOCP_LUT_CASES8(56)
#undef GOCP_LUT_CASES8
#undef GOCP_LUT_CASE
#define GOCP_TERM_CASE(XLV) \
  case 64 + XLV: tiled_terms<R, XLV>(gs + g0, cn, zs, ws, k0, o, ao, tl, mk, acc); break;
          GOCP_TERM_CASE(0) GOCP_TERM_CASE(1) GOCP_TERM_CASE(2) GOCP_TERM_CASE(3)
          GOCP_TERM_CASE(4) GOCP_TERM_CASE(5) GOCP_TERM_CASE(6) GOCP_TERM_CASE(7)
#undef GOCP_TERM_CASE
          default: break;
        }
      }
      if (pc == a.n_pieces - 1) {
        // the last piece has x >> LB = 0: tl is the own tile.  A zero own
        // octet adds nothing to the diagonal part or to the energy.
        C_t<R> res[kAmpsH];
        if (!octet_live(mk, o)) {
#pragma unroll
          for (int i = 0; i < kAmpsH; ++i) {
            res[i] = acc[i];
            acc[i] = cmake<R>(0, 0);
          }
        } else {
          R dr[kAmpsH], dc[kAmpsH], di[kAmpsH], dd[kAmpsH];
#pragma unroll
          for (int i = 0; i < kAmpsH; ++i) dr[i] = dc[i] = di[i] = dd[i] = R(0);
          sum_terms8<R>(a.dz, a.dw, 0, a.nd_mid, k0, dr, dc, true);
          sum_terms8<R>(a.dz, a.dw, a.nd_mid, a.nd, k0, di, dd, false);
          C_t<R> own[kAmpsH];
          tile_octet<R>(tl, ao, own);
          double2 v = s_v[o];
#pragma unroll
          for (int i = 0; i < kAmpsH; ++i) {
            const C_t<R> p = own[i];
            const double pp = (double)p.x * p.x + (double)p.y * p.y;
            v.x += pp;
            v.y += (double)p.x * acc[i].x + (double)p.y * acc[i].y + ((double)dr[i] - (double)dc[i]) * pp;
            const R d0 = dr[i] - dc[i] + idr;
            res[i] = cmake<R>(acc[i].x + d0 * p.x - di[i] * p.y, acc[i].y + d0 * p.y + di[i] * p.x);
            acc[i] = cmake<R>(0, 0);
          }
          s_v[o] = v;
        }
        C_t<R>* dst = a.out + k0;
        // streaming stores (evict-first), so that the output does not push
        // the source state out of L2
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
    }
    __syncwarp();
    if ((threadIdx.x & 31u) == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(empty_s + 8u * st) : "memory");
    if (++st == (uint32_t)S) {
      st = 0;
      ph ^= 1u;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_abort) {
    atomicOr(a.err, kErrStageTimeout);
    // let the copies this block started land before its shared memory goes
    // (always with the full limit, whatever a.wait_ns is)
    for (uint32_t j = it; j < s_next; ++j) mbar_wait(full_s + 8u * (j % S), (j / S) & 1u, kWaitNs);
  }
  // (a normal exit consumed every issued item: nothing is in flight)
  const double v[2] = {s_v[threadIdx.x].x, s_v[threadIdx.x].y};
  if (a.partials &&
      block_grid_sum<2, NT>(v, a.partials, a.counter, gridDim.x, blockIdx.x, a.scal + 1, tot)) {
    if (threadIdx.x == 0) a.scal[0] = a.identity + tot[1] / tot[0];
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_fn(EncodeTiled* out) {
  static std::mutex mu;
  static EncodeTiled fn = nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDriverEntryPointByVersion(cuTensorMapEncodeTiled)");
    if (q != cudaDriverEntryPointSuccess || !p) return fail(GOCP_ECUDA, "cuTensorMapEncodeTiled is not available");
    fn = reinterpret_cast<EncodeTiled>(p);
  }
  *out = fn;
  return GOCP_OK;
}

// Shared-memory opt-in, once per device and precision.
template <typename R>
int smem_optin(int device) {
  static std::mutex mu;
  static std::vector<bool> done;
  std::lock_guard<std::mutex> lk(mu);
  if (device >= (int)done.size()) done.resize(device + 1, false);
  if (!done[device]) {
    cudaError_t e = cudaFuncSetAttribute(k_apply_h_tiled<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tiled_smem<R>());
    if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_apply_h_tiled)");
    done[device] = true;
  }
  return GOCP_OK;
}

// Fraction of nonzero amplitudes up to which the scatter kernel takes a
// state (GOCP_SPARSE_FRAC; 0 keeps every state on the staged kernel; the
// amplitude list holds a quarter of the state at most).
// Limit of a staging wait in the staged kernel: GOCP_STAGE_WAIT_NS, default
// kWaitNs.  0 makes every staging wait give up at once (the kernel flags it
// and returns), which lets a test drive that path.
uint64_t stage_wait_ns() {
  const char* e = std::getenv("GOCP_STAGE_WAIT_NS");
  if (!e || !*e) return kWaitNs;
  const long long v = std::atoll(e);
  return v < 0 ? kWaitNs : (uint64_t)v;
}

double sparse_frac() {
  const char* e = std::getenv("GOCP_SPARSE_FRAC");
  if (!e || !*e) return 0.125;
  const double f = std::atof(e);
  return f < 0.0 ? 0.0 : (f > 0.25 ? 0.25 : f);
}

template <typename R>
int launch_tiled(const DevTables& t, const LiveOctets& lv, int sm_count, const void* psi, void* hpsi,
                 double identity, double* partials, unsigned int* counter, unsigned int* tile_counter, double* scal,
                 int32_t* err, cudaStream_t st) {
  constexpr int LB = TiledBits<R>::LB;
  if (t.n_pieces <= 0 || t.n < LB) return fail(GOCP_EINVAL, "problem has no tiled H psi form");
  if ((reinterpret_cast<uintptr_t>(psi) & 15u) || (reinterpret_cast<uintptr_t>(hpsi) & 15u))
    return fail(GOCP_EINVAL, "states must be 16-byte aligned");
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  int rc;
  EncodeTiled enc;
  if ((rc = encode_fn(&enc)) || (rc = smem_optin<R>(device))) return rc;
  // the state as rows of 128 bytes: 32 floats (complex64) or 16 doubles
  CUtensorMap map;
  const cuuint64_t rows = ((cuuint64_t)1 << t.n) * sizeof(C_t<R>) / 128u;
  const cuuint64_t dims[2] = {128u / sizeof(R), rows};
  const cuuint64_t strides[1] = {128u};
  const cuuint32_t kRows = tile_bytes<R>() / 128u;
  const cuuint32_t box[2] = {(cuuint32_t)(128u / sizeof(R)), kRows < 256u ? kRows : 256u};
  const cuuint32_t estr[2] = {1u, 1u};
  CUresult cr = enc(&map, sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                    const_cast<void*>(psi), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(GOCP_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")");
  const uint32_t flag_words = ((1u << (t.n - LB)) + 31u) / 32u;
  if ((rc = cuda_status(cudaMemsetAsync(t.tflags, 0, flag_words * sizeof(uint32_t), st), "clear tile flags")) ||
      (rc = octet_mask(sizeof(R) == 4 ? GOCP_C64 : GOCP_C128, psi, nullptr, t.n, t.octmask, tile_counter, sm_count,
                       st, t.tflags, LB - 3)))
    return rc;
  // states with few nonzero amplitudes: the scatter kernel (the staged one
  // then returns at once); the choice is made on the device from the count
  const double frac = sparse_frac();
  const bool scatter = frac > 0.0 && lv.aidx && lv.toff && t.n_pieces <= kSpMaxPieces;
  const uint32_t max_amps =
      (uint32_t)std::min<double>((double)lv.acap, std::floor(frac * (double)(1ull << t.n)));
  if (scatter) {
    SparseArgs<R> s;
    s.blob = t.tblob;
    s.piece = t.tpiece;
    s.porder = t.tporder;
    s.n_pieces = t.n_pieces;
    s.n = t.n;
    s.psi = reinterpret_cast<const C_t<R>*>(psi);
    s.out = reinterpret_cast<C_t<R>*>(hpsi);
    s.mask = t.octmask;
    s.max_amps = max_amps;
    s.n_offdiag = (uint32_t)(t.G + t.GL);
    s.hbound = t.hbound;
    s.dmax = t.dmax;
    s.wfix = t.twfix;
    s.wscale = t.twscale;
    s.dz = t.dz;
    s.dw = reinterpret_cast<const R*>(t.dw);
    s.nd = t.nd;
    s.nd_mid = t.nd_mid;
    s.identity = identity;
    s.partials = partials;
    s.counter = counter;
    s.tile_counter = tile_counter;
    s.scal = scal;
    if ((rc = sparse_apply_h<R>(s, lv, sm_count, st))) return rc;
  }
  TiledArgs<R> a;
  a.gate = scatter ? lv.alen : nullptr;
  a.gate_max = max_amps;
  a.blob = t.tblob;
  a.piece = t.tpiece;
  a.mask = t.octmask;
  a.tile_counter = tile_counter;
  a.tile_flags = t.tflags;
  a.n_pieces = t.n_pieces;
  a.n = t.n;
  a.dz = t.dz;
  a.dw = reinterpret_cast<const R*>(t.dw);
  a.nd = t.nd;
  a.nd_mid = t.nd_mid;
  a.out = reinterpret_cast<C_t<R>*>(hpsi);
  a.identity = identity;
  a.partials = partials;
  a.counter = counter;
  a.scal = scal;
  a.err = err;
  a.wait_ns = stage_wait_ns();
  const uint64_t ntiles = 1ull << (t.n - LB);
  const int per_sm = sizeof(R) == 4 ? GOCP_TILED_MINB_C64 : 1;
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)std::max(sm_count, 1) * per_sm);
  k_apply_h_tiled<R><<<grid, tiled_threads<R>(), tiled_smem<R>(), st>>>(map, a);
  count_launches(1);
  return cuda_status(cudaGetLastError(), "k_apply_h_tiled");
}

}  // namespace

int octet_mask(int precision, const void* psi, const void* psi2, int n, uint32_t* mask,
               unsigned int* tile_counter, int sm_count, cudaStream_t st, uint32_t* tile_flags, int tile_shift) {
  if (n < 8 || !mask) return fail(GOCP_EINVAL, "octet mask needs n >= 8 and a buffer");
  const uint32_t n_octets = 1u << (n - 3);
  const int grid = (int)std::min<uint32_t>((n_octets + 255u) / 256u, (uint32_t)std::max(sm_count, 1) * 8u);
  if (precision == GOCP_C64)
    k_octet_mask<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float2*>(psi),
                                              reinterpret_cast<const float2*>(psi2), n_octets, mask, tile_counter,
                                              tile_flags, tile_shift);
  else
    k_octet_mask<double><<<grid, 256, 0, st>>>(reinterpret_cast<const double2*>(psi),
                                               reinterpret_cast<const double2*>(psi2), n_octets, mask, tile_counter,
                                               tile_flags, tile_shift);
  count_launches(1);
  return cuda_status(cudaGetLastError(), "k_octet_mask");
}

int tiled_apply_h(const DevTables& t, const LiveOctets& lv, int precision, int sm_count, const void* psi,
                  void* hpsi, double identity, double* partials, unsigned int* counter,
                  unsigned int* tile_counter, double* scal, int32_t* err, cudaStream_t st) {
  return precision == GOCP_C64 ? launch_tiled<float>(t, lv, sm_count, psi, hpsi, identity, partials, counter,
                                                     tile_counter, scal, err, st)
                               : launch_tiled<double>(t, lv, sm_count, psi, hpsi, identity, partials, counter,
                                                      tile_counter, scal, err, st);
}

}  // namespace gocp
