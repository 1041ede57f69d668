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
// Every wait on an mbarrier gives up after kWaitNs of %globaltimer: the block
// then records bit 1 in the error flags, waits (bounded again) for its own
// copies in flight, and leaves the tile loop; results are then undefined and
// gocp_device_errors reports the flag.
#include <cuda.h>

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

// Waits for the phase with the given parity to complete; false after kWaitNs.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 32; ++i)
      if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tma_rows(uint32_t dst, const CUtensorMap* map, int row, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(bar)
      : "memory");
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

// LUT groups of one x & 7 run; k0 = first global index of the thread's
// output octet, ao = tiled_swz of its octet in the tile.
template <typename R, int XL>
__device__ __forceinline__ void tiled_lut(const HLut<R>* ls, int cn, uint32_t k0, uint32_t ao,
                                          const uint8_t* tile, C_t<R> (&acc)[kAmpsH]) {
  for (int g = 0; g < cn; ++g) {
    const HLut<R>& L = ls[g];
    const uint32_t os = ao ^ L.pad0, reg = L.reg;
    const uint32_t code0 = (uint32_t)(__popc(k0 & L.v0) & 1) | ((uint32_t)(__popc(k0 & L.v1) & 1) << 1) |
                           ((uint32_t)(__popc(k0 & L.v2) & 1) << 2) | ((uint32_t)(__popc(k0 & L.z0) & 1) << 3);
    if (reg == 0u) {
      const R val = L.lut16[code0];
      if (val == R(0)) continue;
      C_t<R> src[kAmpsH];
      tile_octet<R>(tile, os, src);
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
      if (!any) continue;
      C_t<R> src[kAmpsH];
      tile_octet<R>(tile, os, src);
#pragma unroll
      for (int i = 0; i < kAmpsH; ++i) {
        acc[i].x += val[i] * src[i ^ XL].x;
        acc[i].y += val[i] * src[i ^ XL].y;
      }
    }
  }
}

// Term-list groups of one x & 7 run.
template <typename R, int XL>
__device__ __forceinline__ void tiled_terms(const TiledGroup* gs, int cn, const uint32_t* zs, const R* ws,
                                            uint32_t k0, uint32_t ao, const uint8_t* tile,
                                            C_t<R> (&acc)[kAmpsH]) {
  for (int g = 0; g < cn; ++g) {
    const TiledGroup& G = gs[g];
    const uint32_t os = ao ^ G.xa;
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

template <typename R>
struct TiledArgs {
  const uint8_t* blob;
  const TiledPiece* piece;
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
};

template <typename R>
__host__ __device__ constexpr uint32_t tile_bytes() {
  return (1u << TiledBits<R>::LB) * (uint32_t)sizeof(C_t<R>);
}

template <typename R>
__host__ __device__ constexpr int tiled_threads() {
  return 1 << (TiledBits<R>::LB - 3);
}

template <typename R>
__host__ __device__ constexpr size_t tiled_smem() {
  return 1024 + 2 * (size_t)tile_bytes<R>() + 2 * (size_t)kTiledBlobBytes;
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
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int s_abort;
  __shared__ double tot[2];
  // stage st: tile at base + st * kTile, blob at base + 2 kTile + st * blob size
  uint8_t* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const uint32_t base_s = smem_addr(base), bar_s = smem_addr(&bar[0]);
  auto tile_s = [&](int st) { return base_s + (uint32_t)st * kTile; };
  auto blob_s = [&](int st) { return base_s + 2u * kTile + (uint32_t)st * kTiledBlobBytes; };
  auto bar_at = [&](int st) { return bar_s + 8u * (uint32_t)st; };

  // items = (tile, piece) pairs of this block; fewer than 2^32 (tiles <= 2^19)
  const uint32_t ntiles = 1u << (a.n - LB);
  const uint32_t my_tiles = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const uint32_t nitems = my_tiles * (uint32_t)a.n_pieces;
  // per-thread energy partials live in shared memory (touched once per tile)
  __shared__ double2 s_v[NT];
  s_v[threadIdx.x] = make_double2(0.0, 0.0);

  if (threadIdx.x == 0) {
    mbar_init(bar_at(0), 1);
    mbar_init(bar_at(1), 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // thread 0: start the copies of item `it` into stage it & 1
  auto issue = [&](uint32_t it) {
    const int st = (int)(it & 1);
    const uint32_t tile = blockIdx.x + (it / (uint32_t)a.n_pieces) * gridDim.x;
    const TiledPiece pc = a.piece[it % (uint32_t)a.n_pieces];
    const uint32_t src = tile ^ pc.xhi;
    mbar_expect_tx(bar_at(st), kTile + pc.bytes);
#pragma unroll
    for (uint32_t c = 0; c < kRows / kBox; ++c)
      tma_rows(tile_s(st) + c * kBox * 128u, &tmap, (int)(src * kRows + c * kBox), bar_at(st));
    if (pc.bytes) bulk_copy(blob_s(st), a.blob + pc.off, pc.bytes, bar_at(st));
  };
  if (threadIdx.x == 0) {
    if (nitems > 0) issue(0);
    if (nitems > 1) issue(1);
  }

  const R idr = (R)a.identity;
  const uint32_t o = threadIdx.x, ao = tiled_swz<R>(o);
  C_t<R> acc[kAmpsH];
#pragma unroll
  for (int i = 0; i < kAmpsH; ++i) acc[i] = cmake<R>(0, 0);
  uint32_t it = 0, tile = blockIdx.x;
  int pc = 0;
  bool aborted = false;
  for (; it < nitems; ++it) {
    const int st = (int)(it & 1);
    const uint32_t k0 = (tile << LB) + o * kAmpsH;
    if (!mbar_wait(bar_at(st), (it >> 1) & 1u)) {
      s_abort = 1;
    } else {
      const uint8_t* tl = base + (uint32_t)st * kTile;
      const uint8_t* bl = base + 2u * kTile + (uint32_t)st * kTiledBlobBytes;
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
#define GOCP_CASE(XLV)                                                   \
  case XLV: tiled_lut<R, XLV>(ls + g0, cn, k0, ao, tl, acc); break;      \
  case 8 + XLV: tiled_terms<R, XLV>(gs + g0, cn, zs, ws, k0, ao, tl, acc); break;
          GOCP_CASE(0) GOCP_CASE(1) GOCP_CASE(2) GOCP_CASE(3)
          GOCP_CASE(4) GOCP_CASE(5) GOCP_CASE(6) GOCP_CASE(7)
#undef GOCP_CASE
          default: break;
        }
      }
      if (pc == a.n_pieces - 1) {
        // the last piece has x >> LB = 0: tl is the own tile
        R dr[kAmpsH], dc[kAmpsH], di[kAmpsH], dd[kAmpsH];
#pragma unroll
        for (int i = 0; i < kAmpsH; ++i) dr[i] = dc[i] = di[i] = dd[i] = R(0);
        sum_terms8<R>(a.dz, a.dw, 0, a.nd_mid, k0, dr, dc, true);
        sum_terms8<R>(a.dz, a.dw, a.nd_mid, a.nd, k0, di, dd, false);
        C_t<R> own[kAmpsH];
        tile_octet<R>(tl, ao, own);
        C_t<R> res[kAmpsH];
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
        C_t<R>* dst = a.out + k0;
        if (sizeof(R) == 4) {
          float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
          for (int q = 0; q < kAmpsH / 2; ++q)
            d4[q] = make_float4((float)res[2 * q].x, (float)res[2 * q].y, (float)res[2 * q + 1].x,
                                (float)res[2 * q + 1].y);
        } else {
#pragma unroll
          for (int q = 0; q < kAmpsH; ++q) dst[q] = res[q];
        }
      }
    }
    __syncthreads();   // stage st is free again
    if (s_abort) {
      aborted = true;
      break;
    }
    if (threadIdx.x == 0 && it + 2u < nitems) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(it + 2);
    }
    if (++pc == a.n_pieces) {
      pc = 0;
      tile += gridDim.x;
    }
  }
  if (aborted && threadIdx.x == 0) {
    atomicOr(a.err, kErrStageTimeout);
    // let the copies this block started land before its shared memory goes
    for (uint32_t j = it; j < nitems && j < it + 2u; ++j) mbar_wait(bar_at((int)(j & 1)), (j >> 1) & 1u);
  }
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

template <typename R>
int launch_tiled(const DevTables& t, int sm_count, const void* psi, void* hpsi, double identity,
                 double* partials, unsigned int* counter, double* scal, int32_t* err, cudaStream_t st) {
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
  TiledArgs<R> a;
  a.blob = t.tblob;
  a.piece = t.tpiece;
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
  const uint64_t ntiles = 1ull << (t.n - LB);
  const int per_sm = sizeof(R) == 4 ? GOCP_TILED_MINB_C64 : 1;
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)std::max(sm_count, 1) * per_sm);
  k_apply_h_tiled<R><<<grid, tiled_threads<R>(), tiled_smem<R>(), st>>>(map, a);
  count_launches(1);
  return cuda_status(cudaGetLastError(), "k_apply_h_tiled");
}

}  // namespace

int tiled_apply_h(const DevTables& t, int precision, int sm_count, const void* psi, void* hpsi,
                  double identity, double* partials, unsigned int* counter, double* scal, int32_t* err,
                  cudaStream_t st) {
  return precision == GOCP_C64
             ? launch_tiled<float>(t, sm_count, psi, hpsi, identity, partials, counter, scal, err, st)
             : launch_tiled<double>(t, sm_count, psi, hpsi, identity, partials, counter, scal, err, st);
}

}  // namespace gocp
