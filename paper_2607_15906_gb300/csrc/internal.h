// Internal declarations shared by the host builder, the C ABI, the kernels'
// launchers and the request server.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "gocp.h"

typedef struct CUstream_st* cudaStream_t;

namespace gocp {

// ------------------------------------------------------------ errors

// Records `msg` as the calling thread's last error and returns `code`.
int fail(int code, const std::string& msg);
// Returns GOCP_OK after a CUDA call succeeded, else records and returns GOCP_ECUDA.
int cuda_status(int cuda_err, const char* what);
void count_launches(int64_t n);

// Kernel timing (gocp_profile_*): brackets one launch with an event pair on
// its stream while profiling is enabled.
struct ProfScope {
  ProfScope(int kind, void* stream, int launches = 1);   // `launches` kernels between the events
  ~ProfScope();
  int kind;
  void* stream;
  void* start;
  int launches;
};

// ------------------------------------------------------------ exact sums

// Kulisch-style fixed-point accumulator spanning every finite double: each
// added value is placed exactly, and round() returns the correctly rounded
// (half-even) double nearest to the exact sum.
class ExactSum {
 public:
  ExactSum() { clear(); }
  void clear();
  void add(double v);
  double round() const;

 private:
  static constexpr int kLimbs = 70;     // 32-bit digits in signed 64-bit cells
  static constexpr int kOffset = 1088;  // bit index of 2^0
  static constexpr int kMinBit = 14;    // bit index of 2^-1074
  void normalize(int64_t* l) const;
  int64_t limb_[kLimbs];
  int64_t adds_;
  double special_;                      // sum of non-finite inputs
  bool has_special_;
};

// ------------------------------------------------------------ host tables

struct PauliTerms {          // sum_t coeff * i^phase * X^x Z^z
  int n = 0;
  std::vector<uint32_t> x, z;
  std::vector<uint8_t> phase;
  std::vector<double> coeff;
  size_t size() const { return x.size(); }
};

struct Pool {
  std::vector<int64_t> off;   // size M+1
  std::vector<uint32_t> x, z;
  std::vector<uint8_t> phase;
  std::vector<double> coeff;
  std::vector<int32_t> family;   // -1 before colouring
  int n_families = 0;
  int size() const { return off.empty() ? 0 : (int)off.size() - 1; }
};

// Ladder-operator strings of an encoding |n> -> |beta n> over GF(2):
//   a_j = 1/2 X^x Z^zp - 1/2 X^x Z^(zp^ze),  a+_j = 1/2 X^x Z^zp + 1/2 X^x Z^(zp^ze).
struct Encoding {
  int n = 0;
  std::vector<uint32_t> beta_rows;     // row j of beta as a mask
  std::vector<uint32_t> inv_rows;      // row j of beta^-1
  std::vector<uint32_t> x, zp, ze;     // per mode
  uint32_t encode(uint32_t occupation) const;   // qubit basis state of an occupation
  uint32_t decode(uint32_t qubits) const;       // occupation of a qubit basis state
};
Encoding make_encoding(int mapping, int n);

int build_hamiltonian(const gocp_build_args& a, PauliTerms& out);
void build_pool(int n, int n_elec, const Encoding& enc, Pool& out);
// Exact per-(x,z) accumulation of raw strings (duplicates summed, zeros and
// |c| < drop removed, sorted by (x, z)); phases folded into real/imag parts
// must already agree per key, else GOCP_EINVAL.
int canonicalize_terms(const std::vector<uint32_t>& x, const std::vector<uint32_t>& z,
                       const std::vector<uint8_t>& ph, const std::vector<double>& c, double drop,
                       int n, PauliTerms& out);
int colour_pool(Pool& pool);   // Algorithm 1; GOCP_EINVAL if weights are not multiples of 1/8

// Compact form of one x-group D(b) = sum_t w_t (-1)^popc(b & z_t) with real
// weights: with z0 = z of the first term and v_1..v_d a basis of the
// differences z_t ^ z0,
//   D(b) = (-1)^popc(b & z0) * lut[phi(b)],  phi(b)_i = popc(b & v_i) & 1,
// where lut[s] = sum_t w_t (-1)^(c_t . s), c_t the coordinates of z_t ^ z0,
// is summed exactly and rounded once.  ok = false when d > kMaxLutRank.
constexpr int kMaxLutRank = 3;
struct LutForm {
  bool ok = false;
  int d = 0;
  uint32_t z0 = 0;
  uint32_t v[kMaxLutRank] = {0, 0, 0};
  double lut[1 << kMaxLutRank] = {0, 0, 0, 0, 0, 0, 0, 0};
};
LutForm lut_form(const uint32_t* z, const double* w, int count);

// ------------------------------------------------------------ device side

struct DeviceTables;   // defined in kernels.cu
struct SectorTables;   // defined in sector.cu

struct Problem {
  int n_qubits = 0, n_elec = -1, mapping = -1, precision = GOCP_C64, device = -1;
  uint32_t ref_index = 0;
  PauliTerms H;
  Pool pool;
  int64_t n_groups = 0;
  double identity = 0.0;   // coefficient of the identity term (set at upload)
  int sm_count = 0;
  DeviceTables* dev = nullptr;
  size_t device_bytes = 0;
  // sector layout (GOCP_BUILD_SECTOR): states hold the D determinants with
  // n_alpha / n_beta electrons
  bool sector = false;
  int n_alpha = 0, n_beta = 0;
  int64_t sector_dim = 0;
  SectorTables* sec = nullptr;
  struct ChainCache* chains = nullptr;   // replayable launch chains (kernels.cu)
};

// A chain of n launches of one kernel whose arguments differ only in an
// int op index (argument jidx, j = 0..n-1, or n-1..0 with reverse), launched
// on `stream` as one replayable CUDA graph that is built on first use and
// cached on the problem (keyed by the kernel, the grid and the bytes of the
// other arguments).  args[i] points to argument i, sizes[i] is its size.
int launch_chain(Problem& p, const void* kernel, unsigned grid, unsigned block, int n, bool reverse,
                 void** args, const size_t* sizes, int nargs, int jidx, void* stream);
void free_chains(Problem& p);

int upload_problem(Problem& p);
void free_device(Problem& p);

// Sector layout (sector.cu): row tables, built after upload_problem, and the
// launchers of the method's steps on D-amplitude states.
int upload_sector(Problem& p);
void free_sector(Problem& p);
// (stream: a cudaStream_t)
int sec_setup(Problem& p, void* psi, const double* d_theta, int n_ops, void* stream);
int sec_taylor_chain(Problem& p, const int32_t* d_ops, int n_ops, void* psi, void* stream);
int sec_apply_h(Problem& p, const void* psi, void* hpsi, bool energy, void* stream);
int sec_pool_grads(Problem& p, const void* psi, const void* hpsi, double* d_grads, void* stream);
int sec_adjoint(Problem& p, const int32_t* d_ops, int n_ops, void* psi, void* lam, double* d_dE, void* stream);
int sec_expand(Problem& p, const void* psi, void* full, void* stream);
int sec_compress(Problem& p, const void* full, void* psi, void* stream);

// ------------------------------------------------------------ batched stages
//
// One launch advances many resident requests (possibly of different sizes
// and Hamiltonians) by one stage.  Each item's block count depends only on
// the item, so its result is the same alone or in any batch.
struct StageItem {
  const Problem* prob = nullptr;
  void* psi = nullptr;             // state (FORWARD, ENERGY, BACKWARD)
  void* lam = nullptr;             // H psi, then lambda (ENERGY, BACKWARD)
  const int32_t* ops = nullptr;    // device ansatz of the request
  const double* theta = nullptr;
  double* coefs = nullptr;         // 6 per op
  int n_ops = 0;
  int j = 0;                       // operator index of this stage
  double* partials = nullptr;      // >= kMaxItemBlocks doubles
  unsigned int* counter = nullptr; // 1, zero between launches
  double* scal = nullptr;          // [0] E [1] <psi|psi> [2] Re<psi|H'psi>
  double* dtheta = nullptr;        // n_ops doubles
  int32_t* err = nullptr;
};
constexpr int kMaxBatchItems = 256;
constexpr int kMaxItemBlocks = 1216;
enum StageKind { STAGE_SETUP = 0, STAGE_FORWARD = 1, STAGE_ENERGY = 2, STAGE_BACKWARD = 3,
                 STAGE_FORWARD_ALL = 4,    // every forward step of the item, one block (on-chip chain)
                 STAGE_BACKWARD_ALL = 5,   // every backward step of the item, one block
                 STAGE_RESIDUAL = 6 };     // lambda <- (H psi - E psi) / <psi|psi> only (E, <psi|psi> in scal)
// Whether H psi of this problem runs the tiled kernels (full layout from 13
// qubits complex64 / 12 complex128): the server then computes a request's
// H psi and energy with dev_apply_h on the problem's own scratch.
bool has_tiled_form(const Problem& p);
// H psi (+ the energy into scalars_ptr(p): E, <psi|psi>, Re<psi|H'psi>) of a
// full-layout problem on `st` (kernels.cu).
int dev_apply_h(Problem& p, const void* psi, void* hpsi, bool energy, cudaStream_t st);
double* scalars_ptr(Problem& p);
// Whether an item of this problem can take the on-chip stage `kind`
// (STAGE_FORWARD_ALL: its state fits one block's shared memory;
// STAGE_BACKWARD_ALL: its two states do).
bool stage_onchip(const Problem& p, int kind);
// Launches one batched stage over items[0..n) of one precision.  host_desc /
// dev_desc: a pinned host and a device buffer of >= batch_desc_bytes(n)
// bytes used to ship the item descriptors; they must stay untouched until
// the launch completes.
size_t batch_desc_bytes(int n);
int launch_stage(int kind, const StageItem* items, int n, int precision, void* host_desc,
                 void* dev_desc, void* stream, int64_t* launches);

}  // namespace gocp

struct gocp_problem {
  gocp::Problem p;
};
