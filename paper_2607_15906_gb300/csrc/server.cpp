// Continuous-batching request server for energy + dE/dtheta solves.
//
// A worker thread owns one CUDA stream.  Each tick it admits queued requests
// while slots and memory allow, then advances every resident request with
// one batched launch per stage kind and precision:
//   SETUP     |psi> = |ref>, Taylor coefficients of the ansatz
//   FORWARD   psi <- T(theta_j A_j) psi, up to 8 steps a tick     (Eq. 5, 6)
//   ENERGY    lambda <- H psi, E (Eq. 1), lambda <- (H - E) psi / <psi|psi>
//             (from the tile size on: the problem's tiled H psi, per request)
//   BACKWARD  adjoint step j: psi <- T_j^-1 psi, dE_j, lambda <- T_j^+ lambda,
//             up to 8 steps a tick
// A request whose state fits one block's shared memory (up to 14 qubits
// complex64, 13 complex128) takes its whole forward chain in one block
// (FORWARD_ALL), and, when its two states fit, its whole backward sweep
// (BACKWARD_ALL): such a request can finish within the tick that admits it.
// Requests that arrive while others are on the GPU join at the next tick;
// a finished request frees its slot and its memory at once.  Each request
// holds its two states either in one power-of-two block of a buddy-allocated
// arena reserved at creation (hbm_budget_bytes > 0), or (hbm_budget_bytes ==
// 0) in memory taken from a stream-ordered CUDA memory pool when it is
// admitted: it is admitted only while the device's free memory, plus what the
// pool holds unused, covers its two states and a reserve (admission by free
// device memory).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace gocp {
namespace {

constexpr int kMaxOps = 4096;
constexpr int kOpsPerTick = 8;     // forward/backward stages advanced per tick
constexpr size_t kMinBlock = 1 << 16;

// ------------------------------------------------------------ buddy arena

class Buddy {
 public:
  void init(size_t bytes) {
    top_ = 0;
    while ((kMinBlock << (top_ + 1)) <= bytes) ++top_;
    free_.assign(top_ + 1, {});
    size_t top_size = kMinBlock << top_;
    for (size_t off = 0; off + top_size <= bytes; off += top_size) free_[top_].push_back(off);
    capacity_ = (bytes / top_size) * top_size;
  }
  size_t capacity() const { return capacity_; }
  size_t largest() const { return kMinBlock << top_; }
  static int order_for(size_t bytes) {
    int o = 0;
    while ((kMinBlock << o) < bytes) ++o;
    return o;
  }
  bool alloc(int order, size_t* off) {
    if (order > top_) return false;
    int o = order;
    while (o <= top_ && free_[o].empty()) ++o;
    if (o > top_) return false;
    size_t b = free_[o].back();
    free_[o].pop_back();
    while (o > order) {            // split, keep the lower half
      --o;
      free_[o].push_back(b + (kMinBlock << o));
    }
    *off = b;
    return true;
  }
  void release(int order, size_t off) {
    while (order < top_) {
      size_t buddy = off ^ (kMinBlock << order);
      auto& fl = free_[order];
      auto it = std::find(fl.begin(), fl.end(), buddy);
      if (it == fl.end()) break;
      fl.erase(it);
      off = std::min(off, buddy);
      ++order;
    }
    free_[order].push_back(off);
  }

 private:
  int top_ = 0;
  size_t capacity_ = 0;
  std::vector<std::vector<size_t>> free_;
};

// ------------------------------------------------------------ requests

// Lifecycle, read by pollers under the server mutex.
enum class St { Queued, Active, Done, Cancelled, Failed };
// Progress of an active request, touched by the worker thread only.
enum class Phase { Forward, Backward };

struct Slot {   // per-slot device region
  int32_t* ops;
  double* theta;
  double* coefs;
  double* dtheta;
  double* partials;
  unsigned int* counter;
  double* scal;
  int32_t* err;
};

struct Request {
  uint64_t ticket = 0;
  void* mem = nullptr;      // pool mode: the request's two states
  size_t bytes = 0;         // 2 states
  const Problem* prob = nullptr;
  std::vector<int32_t> ops;
  std::vector<double> theta;
  St st = St::Queued;
  Phase phase = Phase::Forward;
  int j = 0;
  int slot = -1;
  int order = 0;
  size_t off = 0;
  bool cancel = false;
  bool needs_setup = true;
  double E = 0.0;
  std::vector<double> dE;
  int status = GOCP_OK;
  std::string msg;
};

}  // namespace
}  // namespace gocp

using namespace gocp;

struct gocp_server {
  int device = 0;
  cudaStream_t stream = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  Buddy buddy;
  // pool mode (hbm_budget_bytes == 0)
  bool pool_mode = false;
  cudaMemPool_t mpool = nullptr;
  size_t reserve = 0;
  size_t capacity = 0;      // device memory less the reserve
  int max_slots = 0;
  void* slot_mem = nullptr;
  std::vector<Slot> slots;
  std::vector<int> free_slots;
  void* host_desc = nullptr;
  void* dev_desc = nullptr;
  size_t desc_stride = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::vector<Request*> resident;
  std::unordered_map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  gocp_server_stats stats{};
  int fatal = GOCP_OK;
  std::string fatal_msg;
};

namespace {

size_t state_bytes_of(const Problem& p) {
  return ((size_t)1 << p.n_qubits) * (p.precision == GOCP_C64 ? 8u : 16u);
}

void finish(gocp_server* s, Request* r, St st) {
  r->st = st;
  if (r->slot >= 0) {
    s->free_slots.push_back(r->slot);
    r->slot = -1;
  }
  if (r->mem) {   // pool mode: back to the pool once the stream's work on it is done
    cudaFreeAsync(r->mem, s->stream);
    r->mem = nullptr;
    s->stats.arena_in_use -= r->bytes;
  }
  if (!s->pool_mode && r->order >= 0 && r->off != (size_t)-1) {
    s->buddy.release(r->order, r->off);
    s->stats.arena_in_use -= kMinBlock << r->order;
    r->off = (size_t)-1;
  }
  if (st == St::Done) ++s->stats.completed;
  if (st == St::Cancelled) ++s->stats.cancelled;
}

// Device memory a pool-mode request may still take: free device memory plus
// what the server's pool holds unused, less the reserve.
size_t pool_available(gocp_server* s) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  uint64_t reserved = 0, used = 0;
  cudaMemPoolGetAttribute(s->mpool, cudaMemPoolAttrReservedMemCurrent, &reserved);
  cudaMemPoolGetAttribute(s->mpool, cudaMemPoolAttrUsedMemCurrent, &used);
  const size_t avail = free_b + (size_t)(reserved > used ? reserved - used : 0);
  return avail > s->reserve ? avail - s->reserve : 0;
}

// Admits queued requests (FIFO with a short look-ahead so that one large
// request does not block smaller ones behind it).  Called with mu held, on
// the worker thread (pool mode allocates on the server stream).
void admit(gocp_server* s) {
  int looked = 0;
  size_t avail = 0;
  bool avail_known = false;
  for (auto it = s->queue.begin(); it != s->queue.end() && looked < 16;) {
    Request* r = *it;
    if (r->cancel) {
      finish(s, r, St::Cancelled);
      it = s->queue.erase(it);
      continue;
    }
    ++looked;
    if (s->free_slots.empty()) break;
    if (s->pool_mode) {
      if (!avail_known) {
        avail = pool_available(s);
        avail_known = true;
      }
      if (r->bytes > avail ||
          cudaMallocFromPoolAsync(&r->mem, r->bytes, s->mpool, s->stream) != cudaSuccess) {
        cudaGetLastError();
        r->mem = nullptr;
        ++it;
        continue;
      }
      avail -= r->bytes;
      s->stats.arena_in_use += r->bytes;
    } else {
      size_t off;
      if (!s->buddy.alloc(r->order, &off)) {
        ++it;
        continue;
      }
      r->off = off;
      s->stats.arena_in_use += kMinBlock << r->order;
    }
    r->slot = s->free_slots.back();
    s->free_slots.pop_back();
    s->stats.arena_peak = std::max(s->stats.arena_peak, s->stats.arena_in_use);
    r->st = St::Active;
    r->phase = Phase::Forward;
    r->j = 0;
    r->needs_setup = true;
    s->resident.push_back(r);
    it = s->queue.erase(it);
  }
  s->stats.max_resident = std::max<uint64_t>(s->stats.max_resident, s->resident.size());
}

StageItem item_for(gocp_server* s, Request* r) {
  const Slot& sl = s->slots[r->slot];
  StageItem it;
  it.prob = r->prob;
  char* base = s->pool_mode ? (char*)r->mem : s->arena + r->off;
  it.psi = base;
  it.lam = base + state_bytes_of(*r->prob);
  it.ops = sl.ops;
  it.theta = sl.theta;
  it.coefs = sl.coefs;
  it.n_ops = (int)r->ops.size();
  it.j = r->j;
  it.partials = sl.partials;
  it.counter = sl.counter;
  it.scal = sl.scal;
  it.dtheta = sl.dtheta;
  it.err = sl.err;
  return it;
}

constexpr int kDescSlotsPerTick = 4 * (2 * kOpsPerTick + 5);

int run_stage(gocp_server* s, int kind, std::vector<StageItem>& items, int* desc_slot,
              int64_t* launches) {
  for (int prec = 0; prec < 2; ++prec) {
    std::vector<StageItem> part;
    for (auto& it : items)
      if (it.prob->precision == prec) part.push_back(it);
    for (size_t b = 0; b < part.size(); b += kMaxBatchItems) {
      int n = (int)std::min<size_t>(kMaxBatchItems, part.size() - b);
      if (*desc_slot >= kDescSlotsPerTick) return fail(GOCP_EINVAL, "descriptor slots exhausted");
      void* hd = (char*)s->host_desc + (size_t)(*desc_slot) * s->desc_stride;
      void* dd = (char*)s->dev_desc + (size_t)(*desc_slot) * s->desc_stride;
      ++*desc_slot;
      int rc = launch_stage(kind, part.data() + b, n, prec, hd, dd, s->stream, launches);
      if (rc) return rc;
    }
  }
  return GOCP_OK;
}

void worker_loop(gocp_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    admit(s);
    // drop cancelled residents
    for (size_t i = 0; i < s->resident.size();) {
      if (s->resident[i]->cancel) {
        finish(s, s->resident[i], St::Cancelled);
        s->resident.erase(s->resident.begin() + i);
        s->cv_done.notify_all();
      } else {
        ++i;
      }
    }
    if (s->resident.empty()) {
      s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
      continue;
    }
    std::vector<Request*> work = s->resident;
    lk.unlock();

    int rc = GOCP_OK;
    int desc_slot = 0;
    int64_t launches = 0;
    // SETUP for newly admitted requests: ansatz upload, |ref>, coefficients
    std::vector<StageItem> items;
    for (Request* r : work)
      if (r->needs_setup) {
        const Slot& sl = s->slots[r->slot];
        size_t n = r->ops.size();
        if (n) {
          cudaMemcpyAsync(sl.ops, r->ops.data(), n * 4, cudaMemcpyHostToDevice, s->stream);
          cudaMemcpyAsync(sl.theta, r->theta.data(), n * 8, cudaMemcpyHostToDevice, s->stream);
        }
        items.push_back(item_for(s, r));
        r->needs_setup = false;
      }
    if (!items.empty()) rc = run_stage(s, STAGE_SETUP, items, &desc_slot, &launches);
    // FORWARD_ALL: requests whose state fits one block's shared memory run
    // their whole forward chain in one block
    if (rc == GOCP_OK) {
      items.clear();
      for (Request* r : work)
        if (r->phase == Phase::Forward && r->j == 0 && !r->ops.empty() &&
            stage_onchip(*r->prob, STAGE_FORWARD_ALL)) {
          items.push_back(item_for(s, r));
          r->j = (int)r->ops.size();
        }
      if (!items.empty()) rc = run_stage(s, STAGE_FORWARD_ALL, items, &desc_slot, &launches);
    }
    // FORWARD: up to kOpsPerTick operators per request
    for (int round = 0; round < kOpsPerTick && rc == GOCP_OK; ++round) {
      items.clear();
      for (Request* r : work)
        if (r->phase == Phase::Forward && r->j < (int)r->ops.size()) {
          items.push_back(item_for(s, r));
          ++r->j;
        }
      if (items.empty()) break;
      rc = run_stage(s, STAGE_FORWARD, items, &desc_slot, &launches);
    }
    // ENERGY for requests whose forward sweep is complete: the batched
    // octet kernel below the tile size; from it on, the problem's own tiled
    // H psi (the scatter kernel for a sector-confined state), one request
    // after the other on this stream, with E and <psi|psi> copied to the
    // request's slot before the next request on the same problem runs
    if (rc == GOCP_OK) {
      items.clear();
      std::vector<StageItem> tiled;
      for (Request* r : work)
        if (r->phase == Phase::Forward && r->j >= (int)r->ops.size()) {
          (has_tiled_form(*r->prob) ? tiled : items).push_back(item_for(s, r));
          r->phase = Phase::Backward;
          r->j = (int)r->ops.size() - 1;
        }
      if (!items.empty()) rc = run_stage(s, STAGE_ENERGY, items, &desc_slot, &launches);
      for (const StageItem& it : tiled) {
        if (rc != GOCP_OK) break;
        Problem& p = const_cast<Problem&>(*it.prob);
        rc = dev_apply_h(p, it.psi, it.lam, true, s->stream);
        if (rc == GOCP_OK)
          rc = cuda_status(cudaMemcpyAsync(it.scal, scalars_ptr(p), 3 * sizeof(double), cudaMemcpyDeviceToDevice,
                                           s->stream),
                           "request energy");
      }
      if (rc == GOCP_OK && !tiled.empty()) rc = run_stage(s, STAGE_RESIDUAL, tiled, &desc_slot, &launches);
    }
    // BACKWARD_ALL: requests whose two states fit one block's shared memory
    // run their whole backward sweep in one block
    if (rc == GOCP_OK) {
      items.clear();
      for (Request* r : work)
        if (r->phase == Phase::Backward && !r->ops.empty() && r->j == (int)r->ops.size() - 1 &&
            stage_onchip(*r->prob, STAGE_BACKWARD_ALL)) {
          items.push_back(item_for(s, r));
          r->j = -1;
        }
      if (!items.empty()) rc = run_stage(s, STAGE_BACKWARD_ALL, items, &desc_slot, &launches);
    }
    // BACKWARD: up to kOpsPerTick adjoint steps
    for (int round = 0; round < kOpsPerTick && rc == GOCP_OK; ++round) {
      items.clear();
      for (Request* r : work)
        if (r->phase == Phase::Backward && r->j >= 0) {
          items.push_back(item_for(s, r));
          --r->j;
        }
      if (items.empty()) break;
      rc = run_stage(s, STAGE_BACKWARD, items, &desc_slot, &launches);
    }
    // results of finished requests
    std::vector<Request*> done;
    for (Request* r : work)
      if (r->phase == Phase::Backward && r->j < 0) {
        const Slot& sl = s->slots[r->slot];
        r->dE.assign(r->ops.size(), 0.0);
        cudaMemcpyAsync(&r->E, sl.scal, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
        if (!r->ops.empty())
          cudaMemcpyAsync(r->dE.data(), sl.dtheta, r->ops.size() * 8, cudaMemcpyDeviceToHost, s->stream);
        done.push_back(r);
      }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (rc == GOCP_OK && e != cudaSuccess) rc = cuda_status(e, "server tick");

    lk.lock();
    ++s->stats.ticks;
    s->stats.launches += launches;
    if (rc != GOCP_OK) {
      s->fatal = rc;
      s->fatal_msg = gocp_last_error();
      for (Request* r : s->resident) {
        r->status = rc;
        r->msg = s->fatal_msg;
        finish(s, r, St::Failed);
      }
      s->resident.clear();
      s->cv_done.notify_all();
      continue;
    }
    for (Request* r : done) {
      finish(s, r, St::Done);
      s->resident.erase(std::find(s->resident.begin(), s->resident.end(), r));
    }
    if (!done.empty()) s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

int gocp_server_create(size_t hbm_budget_bytes, int max_slots, int device, gocp_server** out) {
  if (!out) return fail(GOCP_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_slots < 1 || max_slots > kMaxBatchItems) return fail(GOCP_EINVAL, "max_slots must be in 1..256");
  if (hbm_budget_bytes != 0 && hbm_budget_bytes < kMinBlock) return fail(GOCP_EINVAL, "hbm_budget_bytes too small");
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) return fail(GOCP_ENODEV, "no CUDA device");
  if (device < 0 || device >= count) return fail(GOCP_EINVAL, "device out of range");
  gocp_server* s = new gocp_server();
  s->device = device;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  int rc = GOCP_OK;
  auto bail = [&](int code) {
    if (s->arena) cudaFree(s->arena);
    if (s->mpool) cudaMemPoolDestroy(s->mpool);
    if (s->slot_mem) cudaFree(s->slot_mem);
    if (s->dev_desc) cudaFree(s->dev_desc);
    if (s->host_desc) cudaFreeHost(s->host_desc);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    if (prev >= 0) cudaSetDevice(prev);
    return code;
  };
  if (hbm_budget_bytes == 0) {
    s->pool_mode = true;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if ((rc = cuda_status(cudaMemPoolCreate(&s->mpool, &props), "cudaMemPoolCreate"))) return bail(rc);
    uint64_t keep = UINT64_MAX;   // freed blocks stay in the pool for the next requests
    cudaMemPoolSetAttribute(s->mpool, cudaMemPoolAttrReleaseThreshold, &keep);
    size_t free_b = 0, total_b = 0;
    if ((rc = cuda_status(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo"))) return bail(rc);
    s->reserve = std::max<size_t>((size_t)1 << 30, total_b / 50);
    s->capacity = total_b > s->reserve ? total_b - s->reserve : 0;
    s->arena_bytes = 0;
  } else {
    s->buddy.init(hbm_budget_bytes);
    s->arena_bytes = s->buddy.capacity();
    if ((rc = cuda_status(cudaMalloc((void**)&s->arena, s->arena_bytes), "arena"))) return bail(GOCP_ENOMEM);
  }
  const size_t per_slot = (size_t)kMaxOps * (4 + 8 + 48 + 8) + (size_t)kMaxItemBlocks * 8 + 256;
  if ((rc = cuda_status(cudaMalloc(&s->slot_mem, per_slot * max_slots), "slots"))) return bail(GOCP_ENOMEM);
  cudaMemset(s->slot_mem, 0, per_slot * max_slots);
  s->max_slots = max_slots;
  for (int i = 0; i < max_slots; ++i) {
    char* b = (char*)s->slot_mem + per_slot * i;
    Slot sl;
    sl.partials = (double*)b;
    b += (size_t)kMaxItemBlocks * 8;
    sl.scal = (double*)b;
    b += 64;
    sl.counter = (unsigned int*)b;
    b += 64;
    sl.err = (int32_t*)b;
    b += 128;
    sl.theta = (double*)b;
    b += (size_t)kMaxOps * 8;
    sl.coefs = (double*)b;
    b += (size_t)kMaxOps * 48;
    sl.dtheta = (double*)b;
    b += (size_t)kMaxOps * 8;
    sl.ops = (int32_t*)b;
    s->slots.push_back(sl);
    s->free_slots.push_back(max_slots - 1 - i);
  }
  s->desc_stride = (batch_desc_bytes(kMaxBatchItems) + 255) & ~(size_t)255;
  const size_t desc_total = s->desc_stride * kDescSlotsPerTick;
  if ((rc = cuda_status(cudaMallocHost(&s->host_desc, desc_total), "pinned descriptors"))) return bail(GOCP_ENOMEM);
  if ((rc = cuda_status(cudaMalloc(&s->dev_desc, desc_total), "descriptors"))) return bail(GOCP_ENOMEM);
  if ((rc = cuda_status(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking), "stream"))) return bail(rc);
  s->stats.arena_bytes = s->arena_bytes;
  if (prev >= 0) cudaSetDevice(prev);
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return GOCP_OK;
}

void gocp_server_destroy(gocp_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (auto& kv : s->all)
    if (kv.second->mem) cudaFreeAsync(kv.second->mem, s->stream);
  cudaStreamSynchronize(s->stream);
  if (s->mpool) cudaMemPoolDestroy(s->mpool);
  cudaFree(s->arena);
  cudaFree(s->slot_mem);
  cudaFree(s->dev_desc);
  cudaFreeHost(s->host_desc);
  cudaStreamDestroy(s->stream);
  if (prev >= 0) cudaSetDevice(prev);
  for (auto& kv : s->all) delete kv.second;
  delete s;
}

int gocp_submit(gocp_server* s, const gocp_problem* h, const int32_t* ops, const double* theta,
                int n_ops, uint64_t* ticket) {
  if (!s || !h || !ticket) return fail(GOCP_EINVAL, "NULL argument");
  const Problem& p = h->p;
  if (!p.dev) return fail(GOCP_ENODEV, "problem has no device tables");
  if (p.device != s->device) return fail(GOCP_EINVAL, "problem lives on another device");
  if (p.sector) return fail(GOCP_EINVAL, "the request server takes full-layout problems only");
  if (n_ops < 0 || n_ops > kMaxOps) return fail(GOCP_EINVAL, "n_ops must be in 0..4096");
  if (n_ops > 0 && (!ops || !theta)) return fail(GOCP_EINVAL, "ops/theta is NULL");
  for (int i = 0; i < n_ops; ++i) {
    if (ops[i] < 0 || ops[i] >= p.pool.size()) return fail(GOCP_EINVAL, "ansatz operator out of range");
    if (!std::isfinite(theta[i])) return fail(GOCP_EINVAL, "theta is not finite");
  }
  Request* r = new Request();
  r->prob = &p;
  r->ops.assign(ops, ops + n_ops);
  r->theta.assign(theta, theta + n_ops);
  r->order = Buddy::order_for(2 * state_bytes_of(p));
  r->bytes = (2 * state_bytes_of(p) + 255) & ~(size_t)255;
  r->off = (size_t)-1;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->pool_mode ? r->bytes > s->capacity : (kMinBlock << r->order) > s->buddy.largest()) {
    delete r;
    return fail(GOCP_ENOMEM, "request can never fit the server's device memory");
  }
  if (s->fatal) {
    delete r;
    return fail(s->fatal, "server failed earlier: " + s->fatal_msg);
  }
  r->ticket = s->next_ticket++;
  s->all[r->ticket] = r;
  s->queue.push_back(r);
  ++s->stats.submitted;
  *ticket = r->ticket;
  s->cv_work.notify_all();
  return GOCP_OK;
}

int gocp_poll(gocp_server* s, uint64_t ticket, double* E, double* dE, int64_t timeout_us) {
  if (!s) return fail(GOCP_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(GOCP_EINVAL, "unknown or retired ticket");
  Request* r = it->second;
  auto ready = [&] { return r->st == St::Done || r->st == St::Cancelled || r->st == St::Failed; };
  if (!ready()) {
    if (timeout_us == 0) return fail(GOCP_EAGAIN, "not finished");
    if (timeout_us < 0) {
      s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
      return fail(GOCP_ETIMEDOUT, "not finished within the timeout");
    }
  }
  int rc = GOCP_OK;
  if (r->st == St::Done) {
    if (E) *E = r->E;
    if (dE && !r->dE.empty()) std::memcpy(dE, r->dE.data(), r->dE.size() * 8);
  } else if (r->st == St::Cancelled) {
    rc = fail(GOCP_ECANCELED, "request was cancelled");
  } else {
    rc = fail(r->status ? r->status : GOCP_ECUDA, r->msg);
  }
  s->all.erase(it);
  delete r;
  return rc;
}

int gocp_cancel(gocp_server* s, uint64_t ticket) {
  if (!s) return fail(GOCP_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(GOCP_EINVAL, "unknown or retired ticket");
  it->second->cancel = true;
  s->cv_work.notify_all();
  return GOCP_OK;
}

int gocp_server_get_stats(gocp_server* s, gocp_server_stats* out) {
  if (!s || !out) return fail(GOCP_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->resident = (int)s->resident.size();
  out->queued = (int)s->queue.size();
  return GOCP_OK;
}

}  // extern "C"
