// The C ABI declared in include/gocp.h: argument checks, device selection,
// staging of small host arrays and dispatch to the kernel launchers.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace gocp {

namespace {
thread_local std::string t_last_error;
std::atomic<int64_t> g_launches{0};
}  // namespace

int fail(int code, const std::string& msg) {
  t_last_error = msg;
  return code;
}

int cuda_status(int err, const char* what) {
  if (err == cudaSuccess) return GOCP_OK;
  t_last_error = std::string(what) + ": " + cudaGetErrorString((cudaError_t)err);
  return GOCP_ECUDA;
}

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
struct ProfRecord {
  int kind;
  cudaEvent_t a, b;
  int launches;
};
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
std::vector<ProfRecord> g_prof;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

ProfScope::ProfScope(int k, void* st, int n) : kind(k), stream(st), start(nullptr), launches(n) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  cudaEvent_t a = take_event();
  if (a && cudaEventRecord(a, (cudaStream_t)st) == cudaSuccess) start = a;
}

ProfScope::~ProfScope() {
  if (!start) return;
  cudaEvent_t b = take_event();
  if (!b || cudaEventRecord(b, (cudaStream_t)stream) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.push_back({kind, (cudaEvent_t)start, b, launches});
}

// launchers (kernels.cu)
int ensure_stage(Problem& p, int n_ops);
int32_t* stage_ops_ptr(Problem& p);
double* stage_theta_ptr(Problem& p);
double* dtheta_ptr(Problem& p);
double* scalars_ptr(Problem& p);
double* grads_ptr(Problem& p);
int32_t* selected_ptr(Problem& p);
int32_t* err_ptr(Problem& p);
int dev_setup(Problem& p, void* psi, const double* d_theta, int n_ops, cudaStream_t st);
int dev_taylor_chain(Problem& p, const int32_t* d_ops, int n_ops, void* psi, bool tracked, cudaStream_t st);
int dev_apply_h(Problem& p, const void* psi, void* hpsi, bool energy, cudaStream_t st);
int dev_norm(Problem& p, const void* psi, cudaStream_t st);
int dev_pool_grads(Problem& p, const void* psi, const void* hpsi, double* d_grads, bool mask_current,
                   bool norm_current, cudaStream_t st);
int dev_adjoint(Problem& p, const int32_t* d_ops, int n_ops, void* psi, void* lam, double* d_dE,
                cudaStream_t st);
int dev_select(Problem& p, const double* d_grads, double tie_rel, int32_t* d_out, cudaStream_t st);
int dev_energy_static(Problem& p, const void* psi, void* hpsi, double* out, int mem, cudaStream_t st);

namespace {

struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;   // of the switch to `dev`
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) err = cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int check_problem(const gocp_problem* h) {
  if (!h) return fail(GOCP_EINVAL, "problem is NULL");
  if (!h->p.dev) return fail(GOCP_ENODEV, "problem has no device tables (built with device = -1)");
  return GOCP_OK;
}

int check_mem(int mem) {
  if (mem != GOCP_MEM_HOST && mem != GOCP_MEM_DEVICE) return fail(GOCP_EINVAL, "mem must be GOCP_MEM_HOST or GOCP_MEM_DEVICE");
  return GOCP_OK;
}

size_t state_dim(const Problem& p) { return p.sector ? (size_t)p.sector_dim : (size_t)1 << p.n_qubits; }

size_t state_bytes(const Problem& p) { return state_dim(p) * (p.precision == GOCP_C64 ? 8u : 16u); }

// Makes ops/theta available on the device.  Host arrays are validated and
// copied into the problem's staging buffers.
int stage_ansatz(Problem& p, const int32_t* ops, const double* theta, int n_ops, int mem,
                 cudaStream_t st, const int32_t** d_ops, const double** d_theta) {
  if (n_ops < 0) return fail(GOCP_EINVAL, "n_ops < 0");
  int rc = ensure_stage(p, n_ops);
  if (rc) return rc;
  if (n_ops == 0) {
    *d_ops = stage_ops_ptr(p);
    *d_theta = stage_theta_ptr(p);
    return GOCP_OK;
  }
  if (!ops || !theta) return fail(GOCP_EINVAL, "ops/theta is NULL");
  if (mem == GOCP_MEM_DEVICE) {
    *d_ops = ops;
    *d_theta = theta;
    return GOCP_OK;
  }
  const int m = p.pool.size();
  for (int j = 0; j < n_ops; ++j) {
    if (ops[j] < 0 || ops[j] >= m) return fail(GOCP_EINVAL, "ansatz operator index out of range");
    if (!std::isfinite(theta[j])) return fail(GOCP_EINVAL, "theta is not finite");
  }
  if ((rc = cuda_status(cudaMemcpyAsync(stage_ops_ptr(p), ops, n_ops * sizeof(int32_t),
                                        cudaMemcpyHostToDevice, st), "stage ops")))
    return rc;
  if ((rc = cuda_status(cudaMemcpyAsync(stage_theta_ptr(p), theta, n_ops * sizeof(double),
                                        cudaMemcpyHostToDevice, st), "stage theta")))
    return rc;
  *d_ops = stage_ops_ptr(p);
  *d_theta = stage_theta_ptr(p);
  return GOCP_OK;
}

// Copies n doubles from a device source to `dst` (host or device per mem).
int deliver(const double* src, double* dst, size_t n, int mem, cudaStream_t st) {
  if (n == 0) return GOCP_OK;
  if (src == dst) return GOCP_OK;
  int rc = cuda_status(cudaMemcpyAsync(dst, src, n * sizeof(double),
                                       mem == GOCP_MEM_HOST ? cudaMemcpyDeviceToHost
                                                            : cudaMemcpyDeviceToDevice, st),
                       "copy result");
  if (rc) return rc;
  if (mem == GOCP_MEM_HOST) return cuda_status(cudaStreamSynchronize(st), "synchronise");
  return GOCP_OK;
}

bool valid_drop(double v) { return std::isfinite(v) && v >= 0.0; }

int finish_build(gocp_problem* h, int flags, gocp_problem** out) {
  Problem& p = h->p;
  if (!(flags & GOCP_BUILD_NO_COLOURING) && p.pool.size() > 0) {
    int rc = colour_pool(p.pool);
    if (rc) return rc;
  }
  int64_t groups = 0;
  for (size_t i = 0; i < p.H.size(); ++i)
    if (i == 0 || p.H.x[i] != p.H.x[i - 1]) ++groups;
  p.n_groups = groups;
  if (p.device >= 0) {
    DeviceGuard g(p.device);
    int rc = upload_problem(p);
    if (!rc) rc = upload_sector(p);
    if (rc) {
      free_sector(p);
      free_device(p);
      return rc;
    }
    p.n_groups = groups;
  }
  *out = h;
  return GOCP_OK;
}

int check_device(int device) {
  if (device < -1) return fail(GOCP_EINVAL, "device must be >= -1");
  if (device >= 0) {
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) return fail(GOCP_ENODEV, "no CUDA device available");
    if (device >= count) return fail(GOCP_EINVAL, "device ordinal out of range");
  }
  return GOCP_OK;
}

}  // namespace
}  // namespace gocp

using namespace gocp;

extern "C" {

int gocp_build(const gocp_build_args* a, gocp_problem** out) {
  if (!a || !out) return fail(GOCP_EINVAL, "args/out is NULL");
  if (a->n_orb < 1 || a->n_orb > 16) return fail(GOCP_EINVAL, "n_orb must be in 1..16");
  if (a->n_elec < 0 || a->n_elec > 2 * a->n_orb) return fail(GOCP_EINVAL, "n_elec must be in 0..2*n_orb");
  if (a->mapping != GOCP_JW && a->mapping != GOCP_BK) return fail(GOCP_EINVAL, "mapping must be GOCP_JW or GOCP_BK");
  if (a->precision != GOCP_C64 && a->precision != GOCP_C128) return fail(GOCP_EINVAL, "precision must be GOCP_C64 or GOCP_C128");
  if (!a->h || !a->g) return fail(GOCP_EINVAL, "integrals are NULL");
  if (!valid_drop(a->int_drop) || !valid_drop(a->term_drop)) return fail(GOCP_EINVAL, "drop thresholds must be finite and >= 0");
  if (!std::isfinite(a->e0)) return fail(GOCP_EINVAL, "e0 is not finite");
  const size_t no = a->n_orb;
  for (size_t i = 0; i < no * no; ++i)
    if (!std::isfinite(a->h[i])) return fail(GOCP_EINVAL, "h has a non-finite entry");
  for (size_t i = 0; i < no * no * no * no; ++i)
    if (!std::isfinite(a->g[i])) return fail(GOCP_EINVAL, "g has a non-finite entry");
  int rc = check_device(a->device);
  if (rc) return rc;
  gocp_problem* h = new (std::nothrow) gocp_problem();
  if (!h) return fail(GOCP_ENOMEM, "out of host memory");
  Problem& p = h->p;
  p.n_qubits = 2 * a->n_orb;
  p.n_elec = a->n_elec;
  p.mapping = a->mapping;
  p.precision = a->precision;
  p.device = a->device;
  try {
    if ((rc = build_hamiltonian(*a, p.H))) { delete h; return rc; }
    Encoding enc = make_encoding(a->mapping, p.n_qubits);
    build_pool(p.n_qubits, a->n_elec, enc, p.pool);
    p.ref_index = enc.encode(a->n_elec >= 32 ? 0xffffffffu : ((1u << a->n_elec) - 1u));
    if (a->flags & GOCP_BUILD_SECTOR) {
      // D = C(n_orb, N_a) C(n_orb, N_b), the reference state's electron counts
      auto binom = [](int n, int k) {
        int64_t c = 1;
        for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
        return c;
      };
      p.sector = true;
      p.n_alpha = (a->n_elec + 1) / 2;
      p.n_beta = a->n_elec / 2;
      if (p.n_alpha > a->n_orb) { delete h; return fail(GOCP_EINVAL, "too many alpha electrons for the sector layout"); }
      p.sector_dim = binom(a->n_orb, p.n_alpha) * binom(a->n_orb, p.n_beta);
    }
  } catch (const std::bad_alloc&) {
    delete h;
    return fail(GOCP_ENOMEM, "out of host memory during build");
  }
  rc = finish_build(h, a->flags, out);
  if (rc) delete h;
  return rc;
}

int gocp_build_from_tables(const gocp_table_args* a, gocp_problem** out) {
  if (!a || !out) return fail(GOCP_EINVAL, "args/out is NULL");
  if (a->n_qubits < 1 || a->n_qubits > 32) return fail(GOCP_EINVAL, "n_qubits must be in 1..32");
  if (a->precision != GOCP_C64 && a->precision != GOCP_C128) return fail(GOCP_EINVAL, "precision must be GOCP_C64 or GOCP_C128");
  if (a->n_terms < 0 || (a->n_terms > 0 && (!a->x || !a->z || !a->phase || !a->coeff)))
    return fail(GOCP_EINVAL, "bad term arrays");
  if (a->n_ops < 0 || (a->n_ops > 0 && (!a->op_offsets || !a->op_x || !a->op_z || !a->op_phase || !a->op_coeff)))
    return fail(GOCP_EINVAL, "bad generator arrays");
  const uint32_t lim = a->n_qubits == 32 ? 0xffffffffu : ((1u << a->n_qubits) - 1u);
  if (a->ref_index & ~lim) return fail(GOCP_EINVAL, "ref_index out of range");
  if (a->flags & GOCP_BUILD_SECTOR) return fail(GOCP_EINVAL, "the sector layout needs a problem built from integrals");
  int rc = check_device(a->device);
  if (rc) return rc;
  for (int64_t t = 0; t < a->n_terms; ++t) {
    if ((a->x[t] | a->z[t]) & ~lim) return fail(GOCP_EINVAL, "term mask beyond n_qubits");
    if (a->phase[t] > 3 || !std::isfinite(a->coeff[t])) return fail(GOCP_EINVAL, "bad term phase/coeff");
  }
  gocp_problem* h = new (std::nothrow) gocp_problem();
  if (!h) return fail(GOCP_ENOMEM, "out of host memory");
  Problem& p = h->p;
  p.n_qubits = a->n_qubits;
  p.precision = a->precision;
  p.device = a->device;
  p.ref_index = a->ref_index;
  try {
    std::vector<uint32_t> x(a->x, a->x + a->n_terms), z(a->z, a->z + a->n_terms);
    std::vector<uint8_t> ph(a->phase, a->phase + a->n_terms);
    std::vector<double> c(a->coeff, a->coeff + a->n_terms);
    if ((rc = canonicalize_terms(x, z, ph, c, 0.0, p.n_qubits, p.H))) { delete h; return rc; }
    p.pool.off.push_back(0);
    for (int k = 0; k < a->n_ops; ++k) {
      int64_t b = a->op_offsets[k], e = a->op_offsets[k + 1];
      if (b < 0 || e < b || (k == 0 && b != 0)) { delete h; return fail(GOCP_EINVAL, "op_offsets must start at 0 and not decrease"); }
      std::vector<uint32_t> ox, oz;
      std::vector<uint8_t> op;
      std::vector<double> oc;
      for (int64_t s = b; s < e; ++s) {
        if ((a->op_x[s] | a->op_z[s]) & ~lim) { delete h; return fail(GOCP_EINVAL, "generator mask beyond n_qubits"); }
        if (a->op_phase[s] > 3 || !std::isfinite(a->op_coeff[s])) { delete h; return fail(GOCP_EINVAL, "bad generator phase/coeff"); }
        ox.push_back(a->op_x[s]);
        oz.push_back(a->op_z[s]);
        op.push_back(a->op_phase[s]);
        oc.push_back(a->op_coeff[s]);
      }
      PauliTerms g;
      if ((rc = canonicalize_terms(ox, oz, op, oc, 0.0, p.n_qubits, g))) { delete h; return rc; }
      if (g.size() == 0) { delete h; return fail(GOCP_EINVAL, "a generator sums to zero"); }
      for (size_t s = 0; s < g.size(); ++s)
        if (g.x[s] != g.x[0]) { delete h; return fail(GOCP_EINVAL, "a generator must have a single x mask"); }
      if (g.x[0] == 0) { delete h; return fail(GOCP_EINVAL, "a generator must have x != 0"); }
      for (size_t s = 0; s < g.size(); ++s) {
        p.pool.x.push_back(g.x[s]);
        p.pool.z.push_back(g.z[s]);
        p.pool.phase.push_back(g.phase[s]);
        p.pool.coeff.push_back(g.coeff[s]);
      }
      p.pool.off.push_back((int64_t)p.pool.x.size());
    }
    p.pool.family.assign(p.pool.size(), -1);
  } catch (const std::bad_alloc&) {
    delete h;
    return fail(GOCP_ENOMEM, "out of host memory during build");
  }
  rc = finish_build(h, a->flags, out);
  if (rc) delete h;
  return rc;
}

int gocp_problem_info(const gocp_problem* h, gocp_info* o) {
  if (!h || !o) return fail(GOCP_EINVAL, "NULL argument");
  const Problem& p = h->p;
  std::memset(o, 0, sizeof(*o));
  o->n_qubits = p.n_qubits;
  o->n_elec = p.n_elec;
  o->mapping = p.mapping;
  o->precision = p.precision;
  o->device = p.dev ? p.device : -1;
  o->pool_size = p.pool.size();
  o->n_families = p.pool.n_families;
  o->ref_index = p.ref_index;
  o->n_terms = (int64_t)p.H.size();
  o->n_groups = p.n_groups;
  o->n_pool_strings = (int64_t)p.pool.x.size();
  o->device_bytes = p.device_bytes;
  o->state_dim = (int64_t)state_dim(p);
  o->sector = p.sector ? 1 : 0;
  o->n_alpha = p.n_alpha;
  o->n_beta = p.n_beta;
  return GOCP_OK;
}

int gocp_export_terms(const gocp_problem* h, uint32_t* x, uint32_t* z, uint8_t* phase, double* coeff) {
  if (!h) return fail(GOCP_EINVAL, "problem is NULL");
  const PauliTerms& t = h->p.H;
  if (x) std::memcpy(x, t.x.data(), t.size() * 4);
  if (z) std::memcpy(z, t.z.data(), t.size() * 4);
  if (phase) std::memcpy(phase, t.phase.data(), t.size());
  if (coeff) std::memcpy(coeff, t.coeff.data(), t.size() * 8);
  return GOCP_OK;
}

int gocp_export_pool(const gocp_problem* h, int64_t* off, uint32_t* x, uint32_t* z, uint8_t* phase,
                     double* coeff, int32_t* family) {
  if (!h) return fail(GOCP_EINVAL, "problem is NULL");
  const Pool& p = h->p.pool;
  const size_t s = p.x.size();
  if (off && !p.off.empty()) std::memcpy(off, p.off.data(), p.off.size() * 8);
  if (x) std::memcpy(x, p.x.data(), s * 4);
  if (z) std::memcpy(z, p.z.data(), s * 4);
  if (phase) std::memcpy(phase, p.phase.data(), s);
  if (coeff) std::memcpy(coeff, p.coeff.data(), s * 8);
  if (family) std::memcpy(family, p.family.data(), p.family.size() * 4);
  return GOCP_OK;
}

void gocp_problem_free(gocp_problem* h) {
  if (!h) return;
  if (h->p.sec || h->p.chains) {
    DeviceGuard g(h->p.device);
    free_sector(h->p);
    free_chains(h->p);
  }
  free_device(h->p);
  delete h;
}

int gocp_exact_sum(const double* v, int64_t n, double* out) {
  if (!out || n < 0 || (n > 0 && !v)) return fail(GOCP_EINVAL, "bad arguments");
  ExactSum s;
  for (int64_t i = 0; i < n; ++i) s.add(v[i]);
  *out = s.round();
  return GOCP_OK;
}

size_t gocp_state_bytes(const gocp_problem* h) { return h ? state_bytes(h->p) : 0; }

int gocp_reference_state(const gocp_problem* h, void* psi, void* stream) {
  int rc = check_problem(h);
  if (rc) return rc;
  if (!psi) return fail(GOCP_EINVAL, "psi is NULL");
  Problem& p = const_cast<Problem&>(h->p);
  DeviceGuard g(p.device);
  if (p.sector) return sec_setup(p, psi, nullptr, 0, stream);
  return dev_setup(p, psi, nullptr, 0, (cudaStream_t)stream);
}

int gocp_prepare_state(const gocp_problem* h, const int32_t* ops, const double* theta, int n_ops,
                       int mem, void* psi, void* stream) {
  int rc = check_problem(h);
  if (rc || (rc = check_mem(mem))) return rc;
  if (!psi) return fail(GOCP_EINVAL, "psi is NULL");
  Problem& p = const_cast<Problem&>(h->p);
  DeviceGuard g(p.device);
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t* d_ops;
  const double* d_theta;
  if ((rc = stage_ansatz(p, ops, theta, n_ops, mem, st, &d_ops, &d_theta))) return rc;
  if (p.sector) {
    if ((rc = sec_setup(p, psi, d_theta, n_ops, st))) return rc;
    return sec_taylor_chain(p, d_ops, n_ops, psi, st);
  }
  if ((rc = dev_setup(p, psi, d_theta, n_ops, st))) return rc;
  return dev_taylor_chain(p, d_ops, n_ops, psi, true, st);
}

int gocp_taylor_step(const gocp_problem* h, int op, double theta, void* psi, void* stream) {
  int rc = check_problem(h);
  if (rc) return rc;
  if (!psi) return fail(GOCP_EINVAL, "psi is NULL");
  Problem& p = const_cast<Problem&>(h->p);
  DeviceGuard g(p.device);
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t* d_ops;
  const double* d_theta;
  int32_t ops[1] = {op};
  double th[1] = {theta};
  if ((rc = stage_ansatz(p, ops, th, 1, GOCP_MEM_HOST, st, &d_ops, &d_theta))) return rc;
  if (p.sector) {
    if ((rc = sec_setup(p, nullptr, d_theta, 1, st))) return rc;
    return sec_taylor_chain(p, d_ops, 1, psi, st);
  }
  if ((rc = dev_setup(p, nullptr, d_theta, 1, st))) return rc;
  return dev_taylor_chain(p, d_ops, 1, psi, false, st);   // psi is the caller's: no mask
}

int gocp_apply_h(const gocp_problem* h, const void* psi, void* hpsi, void* stream) {
  int rc = check_problem(h);
  if (rc) return rc;
  if (!psi || !hpsi || psi == hpsi) return fail(GOCP_EINVAL, "psi/hpsi NULL or aliased");
  Problem& p = const_cast<Problem&>(h->p);
  DeviceGuard g(p.device);
  if (p.sector) return sec_apply_h(p, psi, hpsi, false, stream);
  return dev_apply_h(p, psi, hpsi, false, (cudaStream_t)stream);
}

int gocp_sector_expand(const gocp_problem* h, const void* psi, void* full, void* stream) {
  int rc = check_problem(h);
  if (rc) return rc;
  if (!psi || !full) return fail(GOCP_EINVAL, "psi/full is NULL");
  Problem& p = const_cast<Problem&>(h->p);
  DeviceGuard g(p.device);
  return sec_expand(p, psi, full, stream);
}

int gocp_sector_compress(const gocp_problem* h, const void* full, void* psi, void* stream) {
  int rc = check_problem(h);
  if (rc) return rc;
  if (!psi || !full) return fail(GOCP_EINVAL, "psi/full is NULL");
  Problem& p = const_cast<Problem&>(h->p);
  DeviceGuard g(p.device);
  return sec_compress(p, full, psi, stream);
}

int gocp_energy(const gocp_problem* h, const void* psi, void* hpsi, double* out, int mem, void* stream) {
  int rc = check_problem(h);
  if (rc || (rc = check_mem(mem))) return rc;
  if (!psi || !hpsi || psi == hpsi || !out) return fail(GOCP_EINVAL, "psi/hpsi/out NULL or aliased");
  Problem& p = const_cast<Problem&>(h->p);
  DeviceGuard g(p.device);
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = p.sector ? sec_apply_h(p, psi, hpsi, true, st) : dev_apply_h(p, psi, hpsi, true, st))) return rc;
  return deliver(scalars_ptr(p), out, 2, mem, st);
}

int gocp_energy_static(const gocp_problem* h, const void* psi, void* hpsi, double* out, int mem,
                       void* stream) {
  int rc = check_problem(h);
  if (rc || (rc = check_mem(mem))) return rc;
  Problem& p = const_cast<Problem&>(h->p);
  if (p.sector) return fail(GOCP_EINVAL, "gocp_energy_static takes full-layout problems only");
  if (!psi || !hpsi || psi == hpsi || !out) return fail(GOCP_EINVAL, "psi/hpsi/out NULL or aliased");
  DeviceGuard g(p.device);
  if (g.err != cudaSuccess) return cuda_status(g.err, "cudaSetDevice");
  return dev_energy_static(p, psi, hpsi, out, mem, (cudaStream_t)stream);
}

int gocp_pool_gradients(const gocp_problem* h, const void* psi, const void* hpsi, double* grads,
                        int mem, void* stream) {
  int rc = check_problem(h);
  if (rc || (rc = check_mem(mem))) return rc;
  if (!psi || !hpsi || !grads) return fail(GOCP_EINVAL, "psi/hpsi/grads is NULL");
  Problem& p = const_cast<Problem&>(h->p);
  DeviceGuard g(p.device);
  cudaStream_t st = (cudaStream_t)stream;
  double* dst = mem == GOCP_MEM_DEVICE ? grads : grads_ptr(p);
  if ((rc = p.sector ? sec_pool_grads(p, psi, hpsi, dst, st) : dev_pool_grads(p, psi, hpsi, dst, false, false, st)))
    return rc;
  return deliver(dst, grads, p.pool.size(), mem, st);
}

int gocp_energy_grad(const gocp_problem* h, const int32_t* ops, const double* theta, int n_ops,
                     int mem, void* ws, double* E, double* dE, void* stream) {
  int rc = check_problem(h);
  if (rc || (rc = check_mem(mem))) return rc;
  if (!ws || !E || (n_ops > 0 && !dE)) return fail(GOCP_EINVAL, "ws/E/dE is NULL");
  Problem& p = const_cast<Problem&>(h->p);
  DeviceGuard g(p.device);
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t* d_ops;
  const double* d_theta;
  if ((rc = stage_ansatz(p, ops, theta, n_ops, mem, st, &d_ops, &d_theta))) return rc;
  void* psi = ws;
  void* lam = (char*)ws + state_bytes(p);
  double* d_dE = mem == GOCP_MEM_DEVICE ? dE : dtheta_ptr(p);
  if (p.sector) {
    if ((rc = sec_setup(p, psi, d_theta, n_ops, st)) || (rc = sec_taylor_chain(p, d_ops, n_ops, psi, st)) ||
        (rc = sec_apply_h(p, psi, lam, true, st)) ||
        (n_ops > 0 && (rc = sec_adjoint(p, d_ops, n_ops, psi, lam, d_dE, st))))
      return rc;
  } else {
    if ((rc = dev_setup(p, psi, d_theta, n_ops, st))) return rc;
    if ((rc = dev_taylor_chain(p, d_ops, n_ops, psi, true, st))) return rc;
    if ((rc = dev_apply_h(p, psi, lam, true, st))) return rc;
    if (n_ops > 0 && (rc = dev_adjoint(p, d_ops, n_ops, psi, lam, d_dE, st))) return rc;
  }
  if (mem == GOCP_MEM_DEVICE) {
    return cuda_status(cudaMemcpyAsync(E, scalars_ptr(p), sizeof(double), cudaMemcpyDeviceToDevice, st), "copy E");
  }
  if ((rc = cuda_status(cudaMemcpyAsync(E, scalars_ptr(p), sizeof(double), cudaMemcpyDeviceToHost, st), "copy E")))
    return rc;
  if (n_ops > 0 && (rc = cuda_status(cudaMemcpyAsync(dE, d_dE, n_ops * sizeof(double), cudaMemcpyDeviceToHost, st), "copy dE")))
    return rc;
  return cuda_status(cudaStreamSynchronize(st), "synchronise");
}

int gocp_adapt_step(const gocp_problem* h, const int32_t* ops, const double* theta, int n_ops,
                    int mem, void* ws, double tie_rel, double* out_e, double* grads,
                    int32_t* selected, void* stream) {
  int rc = check_problem(h);
  if (rc || (rc = check_mem(mem))) return rc;
  if (!ws || !out_e || !grads || !selected) return fail(GOCP_EINVAL, "NULL output");
  if (!(tie_rel >= 0.0 && tie_rel < 1.0)) return fail(GOCP_EINVAL, "tie_rel must be in [0, 1)");
  Problem& p = const_cast<Problem&>(h->p);
  DeviceGuard g(p.device);
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t* d_ops;
  const double* d_theta;
  if ((rc = stage_ansatz(p, ops, theta, n_ops, mem, st, &d_ops, &d_theta))) return rc;
  void* psi = ws;
  void* hpsi = (char*)ws + state_bytes(p);
  double* d_grads = mem == GOCP_MEM_DEVICE ? grads : grads_ptr(p);
  if (p.sector) {
    if ((rc = sec_setup(p, psi, d_theta, n_ops, st)) || (rc = sec_taylor_chain(p, d_ops, n_ops, psi, st)) ||
        (rc = sec_apply_h(p, psi, hpsi, true, st)) || (rc = sec_pool_grads(p, psi, hpsi, d_grads, st)))
      return rc;
  } else {
    if ((rc = dev_setup(p, psi, d_theta, n_ops, st))) return rc;
    if ((rc = dev_taylor_chain(p, d_ops, n_ops, psi, true, st))) return rc;
    if ((rc = dev_apply_h(p, psi, hpsi, true, st))) return rc;
    // the chain's octet mask, and <psi|psi> from the energy epilogue just run
    if ((rc = dev_pool_grads(p, psi, hpsi, d_grads, true, true, st))) return rc;
  }
  int32_t* d_sel = mem == GOCP_MEM_DEVICE ? selected : selected_ptr(p);
  if ((rc = dev_select(p, d_grads, tie_rel, d_sel, st))) return rc;
  if (mem == GOCP_MEM_DEVICE) {
    return cuda_status(cudaMemcpyAsync(out_e, scalars_ptr(p), 2 * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy E");
  }
  if ((rc = cuda_status(cudaMemcpyAsync(out_e, scalars_ptr(p), 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "copy E")) ||
      (rc = cuda_status(cudaMemcpyAsync(grads, d_grads, p.pool.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "copy grads")) ||
      (rc = cuda_status(cudaMemcpyAsync(selected, d_sel, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy selection")))
    return rc;
  return cuda_status(cudaStreamSynchronize(st), "synchronise");
}

int gocp_device_errors(const gocp_problem* h, int* flags, void* stream) {
  int rc = check_problem(h);
  if (rc) return rc;
  if (!flags) return fail(GOCP_EINVAL, "flags is NULL");
  Problem& p = const_cast<Problem&>(h->p);
  DeviceGuard g(p.device);
  cudaStream_t st = (cudaStream_t)stream;
  int32_t v = 0;
  if ((rc = cuda_status(cudaMemcpyAsync(&v, err_ptr(p), sizeof(int32_t), cudaMemcpyDeviceToHost, st), "read flags")))
    return rc;
  if ((rc = cuda_status(cudaMemsetAsync(err_ptr(p), 0, sizeof(int32_t), st), "clear flags"))) return rc;
  if ((rc = cuda_status(cudaStreamSynchronize(st), "synchronise"))) return rc;
  *flags = v;
  return GOCP_OK;
}

int gocp_profile_enable(int on) {
  g_prof_on.store(on != 0);
  return GOCP_OK;
}

int gocp_profile_read(int kind, int64_t* launches, double* total_ms) {
  if (kind < 0 || kind >= GOCP_KERNEL_KINDS || !launches || !total_ms)
    return fail(GOCP_EINVAL, "bad profile query");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  int64_t n = 0;
  double ms = 0.0;
  std::vector<ProfRecord> keep;
  int rc = GOCP_OK;
  for (const ProfRecord& r : g_prof) {
    if (r.kind != kind) {
      keep.push_back(r);
      continue;
    }
    float t = 0.0f;
    if (rc == GOCP_OK && cudaEventSynchronize(r.b) == cudaSuccess &&
        cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      ms += t;
      n += r.launches;
    } else {
      rc = fail(GOCP_ECUDA, "event timing failed");
    }
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_prof.swap(keep);
  *launches = n;
  *total_ms = ms;
  return rc;
}

const char* gocp_last_error(void) { return t_last_error.c_str(); }
int64_t gocp_launch_count(void) { return g_launches.load(); }
// The k_apply_h revision names the kernel that profiles/traffic.json was measured on.
const char* gocp_version(void) { return "gocp-gb300 0.2 (sm_103a; k_apply_h_tiled=tiled-tma-r12; k_apply_h_sparse=scatter-fixed-r18; chain=amp-list-ring-4; onchip=smem-chain-2; sector=pair-lists-csr-1; chains=graphs-pdl-2; grads=nonzero-amps-2)"; }

}  // extern "C"
