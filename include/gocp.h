/*
 * gocp.h -- C ABI of the GB300 (sm_103a) GOCP ADAPT-VQE hot path.
 *
 * The method (arxiv 2607.15906) evolves a 2^n complex statevector under
 * qubit-mapped Pauli sums: the Hamiltonian H = sum_p c_p P_p of Eq. (3) and
 * anti-Hermitian excitation generators A_k from an operator pool.  This
 * library implements, on one GPU:
 *   - the host build: integrals -> Eq. (2) -> Jordan-Wigner / Bravyi-Kitaev
 *     Pauli table (Sec. II.A), the singles+doubles pool (Table II) and the
 *     Greedy Operator Commutativity Partitioning of the pool (Sec. III.A,
 *     Algorithm 1);
 *   - matrix-free H psi and the energy <psi|H|psi>/<psi|psi> (Eq. 1);
 *   - the chained fifth-order Taylor propagator (Eq. 5, Eq. 6);
 *   - the pool gradients g_k = <psi|[H, A_k]|psi> = 2 Re <H psi|A_k psi>
 *     (Eq. 4);
 *   - dE/dtheta of the whole ansatz by an adjoint sweep of the Taylor chain;
 *   - a continuous-batching request server for energy+gradient solves.
 *
 * Conventions shared by every entry point
 *   Pauli term (x, z, phase, coeff) = coeff * i^phase * X^x Z^z, with x, z
 *     uint32 bit masks (bit j = qubit j, so n <= 32) and Z applied
 *     first: it maps |b> to coeff * i^phase * (-1)^popcount(b & z) |b ^ x>.
 *   Spin-orbital i = 2p + sigma (sigma 0 alpha, 1 beta) sits on qubit i.
 *   A state is an interleaved complex array of 2^n amplitudes, index bit j =
 *     qubit j: float2 (re, im) for GOCP_C64, double2 for GOCP_C128.
 *   The ansatz applies ops[0] first: psi = T(theta[P-1] A_ops[P-1]) ...
 *     T(theta[0] A_ops[0]) |ref>, T the O(5) Taylor series of exp.
 *   Every call returns a status code (GOCP_OK or a negative GOCP_E*); the
 *     message of the calling thread's last failure is in gocp_last_error().
 *     No call traps the device or throws across the ABI.
 *   Inputs passed by pointer are read (and copied where kept) during the
 *     call; the caller keeps ownership.  Objects returned through ** are
 *     owned by the library until the matching _free / _destroy.
 *   Device buffers (states, workspaces, GOCP_MEM_DEVICE arrays) are
 *     caller-owned device memory on the problem's device.  `stream` is a
 *     cudaStream_t (NULL = legacy default stream); work is enqueued on it.
 *     Calls with GOCP_MEM_HOST outputs synchronise that stream before they
 *     return; GOCP_MEM_DEVICE calls return without synchronising.
 *   Calls that compute on the same problem share the problem's reduction
 *     scratch, so they must be ordered (one stream, or externally
 *     serialised).  Different problems are independent.
 */
#ifndef GOCP_H
#define GOCP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  GOCP_OK = 0,
  GOCP_EINVAL = -1,     /* bad argument; nothing was enqueued */
  GOCP_ENOMEM = -2,     /* host or device allocation failed */
  GOCP_ECUDA = -3,      /* a CUDA runtime call failed */
  GOCP_EAGAIN = -4,     /* result not ready (poll with zero timeout) */
  GOCP_ETIMEDOUT = -5,  /* wait ran out */
  GOCP_ECANCELED = -6,  /* request was cancelled */
  GOCP_ENODEV = -7      /* no device tables (host-only problem) or no GPU */
};
enum { GOCP_JW = 0, GOCP_BK = 1 };          /* qubit mapping, Sec. II.A */
enum { GOCP_C64 = 0, GOCP_C128 = 1 };       /* amplitude precision */
enum { GOCP_MEM_HOST = 0, GOCP_MEM_DEVICE = 1 };
/* gocp_build_args.flags.  GOCP_BUILD_SECTOR (gocp_build only) selects the
 * sector layout: a state holds only the D = C(n_orb, N_a) C(n_orb, N_b)
 * determinants with the reference state's N_a = ceil(n_elec / 2) alpha and
 * N_b = floor(n_elec / 2) beta electrons, row r = rank_a * C(n_orb, N_b) +
 * rank_b (colexicographic ranks of the alpha and beta occupation strings,
 * spin-orbital 2p + s).  H and every pool generator conserve both counts, so
 * each operation of the method maps this subspace to itself: states, E,
 * gradients and dE/dtheta equal the full-layout ones, and H psi equals the
 * full-layout H psi on the sector rows (a term_drop that removes part of a
 * number-conserving set of Pauli terms leaves a small full-layout H psi
 * outside the sector, which this layout does not hold).  Every
 * state argument below then has gocp_state_bytes() = D * (8 or 16) bytes;
 * gocp_sector_expand / _compress convert to and from the 2^n layout.  The
 * request server and gocp_energy_static take full-layout problems only. */
enum { GOCP_BUILD_NO_COLOURING = 1, GOCP_BUILD_SECTOR = 2 };

typedef struct gocp_problem gocp_problem;
typedef struct gocp_server gocp_server;

/* ------------------------------------------------------------------ build */

/* Spatial-orbital integrals of Eq. (2) (h_ijkl read as <ij|kl> = (ik|jl)):
 *   H = e0 + sum_{pq,s} h[p*n+q] a+_{ps} a_{qs}
 *          + 1/2 sum_{pqrs,s,t} g[((p*n+q)*n+r)*n+s] a+_{ps} a+_{rt} a_{st} a_{qs}
 * with g in chemist order (pq|rs) and the 8-fold symmetry of real orbitals.
 * int_drop zeroes integrals with |v| < int_drop before mapping; mapped terms
 * are summed exactly (one rounding per term) and those with |c| < term_drop
 * dropped.  Pool: spin-conserving singles then doubles over occupied
 * spin-orbitals 0..n_elec-1 (Table II counts).  device >= 0 uploads the
 * tables to that CUDA device; device = -1 builds host tables only (export
 * works, compute calls return GOCP_ENODEV). */
typedef struct {
  int n_orb;            /* spatial orbitals; qubits = 2*n_orb, 1..16 */
  int n_elec;           /* electrons, 0..2*n_orb */
  int mapping;          /* GOCP_JW | GOCP_BK */
  int precision;        /* GOCP_C64 | GOCP_C128 */
  const double* h;      /* n_orb^2, row-major, symmetric */
  const double* g;      /* n_orb^4, chemist order */
  double e0;            /* constant energy */
  double int_drop;      /* >= 0 */
  double term_drop;     /* >= 0 */
  int device;           /* CUDA ordinal, or -1 */
  int flags;            /* GOCP_BUILD_* bits */
} gocp_build_args;

/* Build a problem from integrals (Eq. 2 -> Eq. 3, pool, Algorithm 1).
 * Returns GOCP_EINVAL on bad sizes or pointers, GOCP_ENOMEM / GOCP_ECUDA on
 * allocation or upload failure; *out is set only on success. */
int gocp_build(const gocp_build_args* args, gocp_problem** out);

/* Build a problem from caller-supplied Pauli tables (any Hermitian H and
 * any generators).  Terms need not be sorted or unique: duplicates are
 * summed exactly.  Generator k is strings [op_offsets[k], op_offsets[k+1])
 * and must be a single x-mask group with x != 0 (one pair per basis state,
 * as every fermionic excitation is).  ref_index is the reference basis
 * state.  GOCP families are computed unless GOCP_BUILD_NO_COLOURING is set
 * (the commutator test needs generator coefficients that are multiples of
 * 1/8; otherwise GOCP_EINVAL). */
typedef struct {
  int n_qubits;                 /* 1..32 */
  int precision;
  int device;
  int flags;
  int64_t n_terms;
  const uint32_t* x;
  const uint32_t* z;
  const uint8_t* phase;         /* 0..3 */
  const double* coeff;
  int n_ops;
  const int64_t* op_offsets;    /* n_ops + 1, non-decreasing from 0 */
  const uint32_t* op_x;
  const uint32_t* op_z;
  const uint8_t* op_phase;
  const double* op_coeff;
  uint32_t ref_index;
} gocp_table_args;
int gocp_build_from_tables(const gocp_table_args* args, gocp_problem** out);

typedef struct {
  int n_qubits;
  int n_elec;             /* -1 for table-built problems */
  int mapping;            /* -1 for table-built problems */
  int precision;
  int device;             /* -1: host tables only */
  int pool_size;          /* M */
  int n_families;         /* K of Algorithm 1, 0 if not coloured */
  uint32_t ref_index;     /* reference basis state */
  int64_t n_terms;        /* T */
  int64_t n_groups;       /* distinct x masks of H */
  int64_t n_pool_strings;
  size_t device_bytes;    /* device memory held by the problem */
  int64_t state_dim;      /* amplitudes per state: 2^n, or D in the sector layout */
  int sector;             /* 1: sector layout (GOCP_BUILD_SECTOR) */
  int n_alpha, n_beta;    /* sector electron counts (0 in the full layout) */
} gocp_info;
int gocp_problem_info(const gocp_problem* p, gocp_info* out);

/* Copy H's table out, sorted by (x, z) ascending; arrays sized n_terms. */
int gocp_export_terms(const gocp_problem* p, uint32_t* x, uint32_t* z, uint8_t* phase, double* coeff);

/* Copy the pool out: op_offsets (pool_size+1), strings (n_pool_strings,
 * each generator's strings sorted by z), family (pool_size; -1 when not
 * coloured).  Any pointer may be NULL to skip that array. */
int gocp_export_pool(const gocp_problem* p, int64_t* op_offsets, uint32_t* x, uint32_t* z,
                     uint8_t* phase, double* coeff, int32_t* family);

void gocp_problem_free(gocp_problem* p);

/* Correctly rounded (round-half-even) value of the exact sum of v[0..n-1],
 * the summation the builder uses for every Pauli coefficient. */
int gocp_exact_sum(const double* v, int64_t n, double* out);

/* ---------------------------------------------------------------- compute */

/* Bytes of one state: state_dim * (8 for C64, 16 for C128), state_dim =
 * 2^n, or D for the sector layout. */
size_t gocp_state_bytes(const gocp_problem* p);

/* Sector layout only (GOCP_EINVAL otherwise): full <- the 2^n state whose
 * amplitude at the basis state of row r is psi[r] and zero elsewhere
 * (full: 2^n amplitudes of the problem's precision, device memory);
 * compress: psi[r] <- full[basis state of row r], the rest of full ignored. */
int gocp_sector_expand(const gocp_problem* p, const void* psi, void* full, void* stream);
int gocp_sector_compress(const gocp_problem* p, const void* full, void* psi, void* stream);

/* psi <- |ref>. */
int gocp_reference_state(const gocp_problem* p, void* psi, void* stream);

/* psi <- T(theta_{P-1} A_{ops[P-1]}) ... T(theta_0 A_{ops[0]}) |ref>, each T
 * the literal chain of Eq. (6): v_0 = psi, v_m = A v_{m-1},
 * psi' = sum_{m=0..5} theta^m/m! v_m (Eq. 5).  ops/theta are host or device
 * arrays per `mem`; ops must lie in [0, pool_size) (GOCP_EINVAL for host
 * arrays; device arrays are clamped and flagged, see gocp_device_errors).
 * n_ops may be 0.  A chain of several steps on a full-layout state of at
 * most 128 KiB runs in one thread block over shared memory (complex64 by
 * default); the environment variable GOCP_ONCHIP_CHAINS = "off" | "block" |
 * "all" selects the grid kernels only, the one-block form, or that and a
 * thread-block cluster's shared memory for states up to 2 MiB.  Larger
 * states run one launch per step, replayed as a CUDA graph whose steps are
 * joined by programmatic dependencies (GOCP_CHAIN_PDL=0: by full
 * completion).  Every form gives the same state bit for bit. */
int gocp_prepare_state(const gocp_problem* p, const int32_t* ops, const double* theta, int n_ops,
                       int mem, void* psi, void* stream);

/* Apply the Taylor step of pool operator `op` to psi in place. */
int gocp_taylor_step(const gocp_problem* p, int op, double theta, void* psi, void* stream);

/* hpsi <- H psi (Eq. 3), matrix-free.  psi and hpsi must not overlap.
 * Full layout from 13 (complex64) / 12 (complex128) qubits: a state whose
 * nonzero amplitudes are at most GOCP_SPARSE_FRAC (environment, default
 * 0.125, at most 0.25; 0 = never) of 2^n goes through the scatter kernel,
 * which sums the products in 64-bit fixed point (integer adds: the result
 * is the same bit for bit from run to run); other states through the
 * staged kernel (fixed order).  The choice is made on the device from the
 * count of nonzero amplitudes.  With few output tiles the scatter kernel
 * lets up to 64 blocks share a tile (GOCP_SCATTER_PARTS, environment, caps
 * that number; 1 = one block per tile); the result does not depend on it.
 * complex64 adds each fixed-point product as two independent 32-bit
 * counts when H has fewer than 65536 off-diagonal x-groups
 * (GOCP_SCATTER_SPLIT=0: as one 64-bit add with a carry); same result. */
int gocp_apply_h(const gocp_problem* p, const void* psi, void* hpsi, void* stream);

/* hpsi <- H psi, and out[0] = E = Re<psi|H psi>/<psi|psi> (Eq. 1),
 * out[1] = <psi|psi>, both reduced in FP64.  `out` (2 doubles) is host or
 * device memory per `mem`. */
int gocp_energy(const gocp_problem* p, const void* psi, void* hpsi, double* out, int mem,
                void* stream);

/* grads[k] = 2 Re <H psi|A_k psi> / <psi|psi> for every pool operator k
 * (Eq. 4 on the normalised state), with hpsi = H psi from gocp_energy or
 * gocp_apply_h.  Operators are evaluated family by family (GOCP order);
 * results are stored in pool order.  grads has pool_size doubles. */
int gocp_pool_gradients(const gocp_problem* p, const void* psi, const void* hpsi, double* grads,
                        int mem, void* stream);

/* E(theta) and dE/dtheta_j for j < n_ops by an adjoint sweep of the Taylor
 * chain: forward prepare, H psi, lambda = (H - E) psi / <psi|psi>, then for
 * j = P-1..0 un-compute psi_j exactly per basis pair, accumulate
 * 2 Re <lambda|T'_j psi_j> and propagate lambda <- T_j^dagger lambda.
 * ws: caller device buffer of >= 2 states (2 * gocp_state_bytes).
 * E (1 double) and dE (n_ops doubles) are host or device per `mem`. */
int gocp_energy_grad(const gocp_problem* p, const int32_t* ops, const double* theta, int n_ops,
                     int mem, void* ws, double* E, double* dE, void* stream);

/* One ADAPT selection step (Sec. II.B): prepare psi(theta) in ws[0],
 * H psi in ws[1], E, all pool gradients and the selected operator
 * (largest |g_k|; values within relative tie_rel of the largest count as
 * ties, lowest index wins).  out_e: 2 doubles (E, <psi|psi>); grads:
 * pool_size doubles; selected: 1 int32.  All per `mem`. */
int gocp_adapt_step(const gocp_problem* p, const int32_t* ops, const double* theta, int n_ops,
                    int mem, void* ws, double tie_rel, double* out_e, double* grads,
                    int32_t* selected, void* stream);

/* H psi and the energy (E, <psi|psi>) like gocp_energy, computed without
 * allocating anything: the reduction scratch is a fixed device array inside
 * this library rather than memory of the problem or of the call.  The paper
 * has no counterpart.  It serves callers that cannot call cudaMalloc at the
 * point where they compute -- a host loop with real-time or no-blocking
 * guarantees (cudaMalloc can block and synchronise the device), or a caller
 * whose device memory is owned by another allocator -- and that pass every
 * input and output themselves (tables built earlier, psi, hpsi, out).
 * It runs the untiled H psi kernel: below the tile size (13 qubits for
 * complex64, 12 for complex128) that is gocp_energy's own kernel and block
 * decomposition, so the results are bit-identical; from the tile size on
 * gocp_energy runs the tiled kernels and the two agree within rounding (the
 * parity tolerances), not bit for bit.
 * Limits: at most 24 qubits (the array holds 8192 block partials, one per
 * 2048-amplitude tile; larger states return GOCP_EINVAL with the numbers);
 * full-layout problems only.  The array (about 128 KiB) is held on every GPU
 * that loads the library until the process exits.  The first call on a
 * device resolves the array's address there (cudaGetSymbolAddress) and keeps
 * it, so make that first call before any stream capture, and make no call
 * after a cudaDeviceReset in the same process.  Every call shares the one
 * array: calls that overlap on the GPU race, so order them on one stream.
 * out: 2 doubles (E, <psi|psi>), host or device per `mem`. */
int gocp_energy_static(const gocp_problem* p, const void* psi, void* hpsi, double* out, int mem,
                       void* stream);

/* Device-side errors flagged since the last call, and clear them.  Bit 0: an
 * op index out of range in a GOCP_MEM_DEVICE ansatz.  Bit 1: a shared-memory
 * staging wait of the staged H psi kernel gave up (after 2 s, or after
 * GOCP_STAGE_WAIT_NS nanoseconds when that environment variable is set, at
 * once when it is 0; the H psi and energy of that call are then undefined,
 * later calls are not affected).  Synchronises `stream`. */
int gocp_device_errors(const gocp_problem* p, int* flags, void* stream);

/* ---------------------------------------------------------------- serving */

/* A request server: a worker thread owns one stream and advances every
 * resident request by one stage per tick with one batched launch per stage
 * kind (forward Taylor op, H psi + energy, adjoint op), admitting queued
 * requests as slots and memory free up (continuous batching).  A request
 * holds 2 states.  Admission:
 *   hbm_budget_bytes == 0: by free device memory -- a queued request is
 *     admitted when the device's free memory (cudaMemGetInfo) plus what the
 *     server's stream-ordered memory pool holds unused covers its two states
 *     and a reserve of max(1 GiB, 2 % of the device), its states are taken
 *     from that pool and returned to it when it finishes;
 *   hbm_budget_bytes > 0: that many bytes are reserved up front as the
 *     state arena (power-of-two buddy blocks).
 * max_slots bounds residency (1..256).  Problems must outlive the requests
 * that name them and must be C64 or C128 problems built on `device`.  The
 * server computes H psi of requests of 13 qubits or more (12 for C128) with
 * the problem's own scratch, so while such requests are queued or running no
 * other call may compute on their problem. */
int gocp_server_create(size_t hbm_budget_bytes, int max_slots, int device, gocp_server** out);
void gocp_server_destroy(gocp_server* s);

/* Queue an energy+gradient request; ops/theta are host arrays copied here.
 * GOCP_ENOMEM if one request can never fit the arena (arena mode). */
int gocp_submit(gocp_server* s, const gocp_problem* p, const int32_t* ops, const double* theta,
                int n_ops, uint64_t* ticket);

/* Wait up to timeout_us (0 = do not wait, <0 = forever) for a request.
 * GOCP_OK: E and dE (n_ops doubles, host) written, ticket retired.
 * GOCP_EAGAIN (timeout 0) / GOCP_ETIMEDOUT: not finished yet.
 * GOCP_ECANCELED: the request was cancelled; ticket retired.
 * GOCP_EINVAL: unknown or already retired ticket. */
int gocp_poll(gocp_server* s, uint64_t ticket, double* E, double* dE, int64_t timeout_us);

/* Cancel a queued or running request (it stops at its next stage). */
int gocp_cancel(gocp_server* s, uint64_t ticket);

typedef struct {
  uint64_t submitted, completed, cancelled;
  uint64_t ticks;               /* worker iterations that launched work */
  uint64_t launches;            /* batched kernel launches */
  uint64_t max_resident;        /* peak concurrent requests */
  size_t arena_bytes, arena_in_use, arena_peak;   /* arena_bytes 0 in free-memory mode */
  int resident, queued;
} gocp_server_stats;
int gocp_server_get_stats(gocp_server* s, gocp_server_stats* out);

/* ---------------------------------------------------------- kernel timing */

/* While enabled, every launch of the kernel kinds below is bracketed by a
 * CUDA event pair recorded on the launching stream.  gocp_profile_read
 * waits for the recorded events of one kind, returns their launch count and
 * summed elapsed milliseconds, and forgets them.  Disabled by default. */
enum { GOCP_KERNEL_APPLY_H = 0, GOCP_KERNEL_TAYLOR = 1, GOCP_KERNEL_POOL_GRAD = 2,
       GOCP_KERNEL_ADJOINT = 3, GOCP_KERNEL_KINDS = 4 };
int gocp_profile_enable(int on);
int gocp_profile_read(int kind, int64_t* launches, double* total_ms);

/* -------------------------------------------------------------- utilities */

const char* gocp_last_error(void);      /* thread-local, never NULL */
int64_t gocp_launch_count(void);        /* kernels launched by this library */
const char* gocp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GOCP_H */
