/*
 * ed.h - C ABI of the GB300 exact-diagonalization library (libed).
 *
 * The library computes the ground-state energy of the tight-binding / Hubbard
 * Hamiltonian
 *     H = -t sum_<ij> sum_sigma (c+_{i sigma} c_{j sigma} + h.c.) + U sum_i n_{i up} n_{i dn}
 * (Siro & Harju, arXiv:1511.00863, Sec. 1 Eq. 1 and the on-site term) in the basis of
 * fixed particle numbers (N_up, N_dn) (Sec. 2.1, Eq. 2) with the Lanczos iteration
 * (Sec. 2.2, Algorithm 1). Everything runs on one CUDA device.
 *
 * Conventions shared by every entry point
 *  - Basis order (Sec. 2.1; the paper leaves the order to its Ref. [Siro 2012]): a
 *    single-species state is an n_sites-bit integer, bit i = site i occupied; states of
 *    one species are ranked in ascending integer order. The two-species index is
 *    rank_up * dim_dn + rank_dn (Sec. 4, Eqs. 5-6).
 *  - Fermion sign: creation operators ordered by ascending site within a species, all up
 *    before all down; a hop c+_i c_j carries (-1)^(particles of the same species strictly
 *    between i and j). The hop matrix element is -t * sign.
 *  - Bonds are an explicit list; a pair listed k times hops with amplitude k*t.
 *  - Vectors passed to the library are DEVICE pointers in the dense layout above, owned by
 *    the caller and never freed by the library; they must be 16-byte aligned and must not
 *    alias each other. Host pointers are named as such.
 *  - Every call is ordered on the caller's CUDA stream (`stream`, a cudaStream_t; NULL =
 *    the legacy default stream). Calls that return host scalars synchronise that stream.
 *  - Objects (ed_basis, ed_lanczos) are bound to the device that was current when they
 *    were created; use them with that device current.
 *  - Errors: a negative ed_status. ed_last_error() gives a message for the calling thread.
 *    No entry point aborts the process or leaves device work running on error.
 */
#ifndef ED_H_
#define ED_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ED_OK = 0,
  ED_BREAKDOWN = 1,          /* b_{j+1} = 0 in Algorithm 1: an invariant subspace was found;
                                success, the energy returned is exact for that subspace */
  ED_ERR_ARG = -1,           /* invalid argument; nothing was launched */
  ED_ERR_OOM = -2,           /* device memory allocation failed */
  ED_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  ED_ERR_TIMEOUT = -4,       /* a bounded device-side wait ran out */
  ED_ERR_NOT_CONVERGED = -5  /* max_steps reached before the convergence test passed;
                                the last estimate is still returned */
} ed_status;

/* Vector precision.
 *  ED_F64         FP64-accurate: FP64 inputs and outputs; the Lanczos vectors are kept as
 *                 int64 fixed point with one FP64 scale per vector (each element rounded to
 *                 2^-(vb) of the vector's largest element, vb >= 53 for lattices with fewer
 *                 than 510 hops per state), hop sums and dot products exact in integers.
 *                 GB300 executes FP64 arithmetic at about 1/70 of its FP32 rate; this path
 *                 runs no FP64 instruction per vector element.
 *  ED_F32         FP32 vectors and FP32 H.v arithmetic; a_j, b_j and the tridiagonal
 *                 eigensolve in FP64. Dot products and norms: each thread accumulates its
 *                 products as a compensated FP32 pair (exact product by FMA, error-free
 *                 sums: the Dot2 scheme of Ogita, Rump & Oishi 2005, about twice FP32
 *                 precision), converted to FP64 once per thread and summed in FP64 across
 *                 threads and CTAs.
 *  ED_F64_NATIVE  FP64 vectors and FP64 arithmetic throughout (the plain method).
 *  ED_C32         complex vectors (interleaved re, im) of FP32 pairs, complex FP32 H.v
 *                 arithmetic; a_j, b_j (real for Hermitian H), dot products and the
 *                 tridiagonal eigensolve in FP64. For lattices with complex amplitudes.
 *  ED_C64         complex vectors of FP64 pairs, FP64 arithmetic throughout.
 * Complex vectors are arrays of dim (re, im) pairs = 2 dim scalars, element i of the basis
 * at scalars 2i, 2i + 1. A real dtype requires a lattice without t_bond; a complex dtype
 * takes either (no t_bond: every amplitude 1). */
typedef enum {
  ED_F64 = 0,
  ED_F32 = 1,
  ED_F64_NATIVE = 2,
  ED_C32 = 3,
  ED_C64 = 4
} ed_dtype;

/* Lattice (Sec. 2.1): n_sites in [1, 32]; bonds is a HOST array [n_bonds][2] of site
 * pairs (i != j, both in range), read during ed_build_basis only. t_bond is NULL (every
 * bond hops with amplitude t, Eq. 1) or a HOST array of n_bonds complex relative
 * amplitudes as (re, im) pairs (2 n_bonds doubles): bond b = (i, j) then contributes
 * -t (tau_b c+_i c_j + conj(tau_b) c+_j c_i) for each spin (the checkerboard lattice's
 * complex hoppings, Sec. 2.1 Fig. 1), and only the complex dtypes apply. */
typedef struct {
  int32_t n_sites;
  int32_t n_bonds;
  const int32_t* bonds;
  const double* t_bond;
} ed_lattice;

/* Model parameters: hopping t (Eq. 1) and on-site interaction U. */
typedef struct {
  double t;
  double U;
} ed_params;

/* Lanczos options (Sec. 2.2).
 *  max_steps  Krylov dimension cap m (1..ED_MAX_STEPS).
 *  tol        stop when |E0(j) - E0(j-1)| <= tol * max(|E0(j)|, 1) (E0(j) = lowest
 *             eigenvalue of T_j); tol <= 0 runs exactly max_steps steps.
 *  reorth     0 = none (Algorithm 1 as printed, two work vectors).
 *             1 = full: the run stores every Lanczos vector f_1..f_m on the device (in the
 *                 run's own storage: FP32, FP64 or int64 fixed point) and, at every step,
 *                 removes from q = w - a_j f_j its components along f_1..f_j by two passes
 *                 of classical Gram-Schmidt; dot products in FP64 (ED_F64_NATIVE),
 *                 compensated FP32 summed in FP64 (ED_F32) or exact integers (ED_F64).
 *             2 = partial (Simon 1984): the level of orthogonality is estimated from the
 *                 a_j, b_j recurrence on the device, and the same passes run only at the
 *                 steps where it exceeds sqrt(eps) (and the step after).
 *             Modes 1 and 2 need (max_steps + 1) stored vectors of device memory (ED_ERR_OOM
 *             otherwise) and apply to the real dtypes only (ED_ERR_ARG for complex ones
 *             and for ed_lanczos_solve_batched). Algorithm 1 itself (Sec. 2.2) has no
 *             reorthogonalisation; without it, copies of converged eigenvalues appear in
 *             T_m after many steps (E0 is unaffected).
 *  seed       SplitMix64 seed of the random start vector when f1 == NULL.
 *  dtype      see ed_dtype; f1 vectors are FP64 for ED_F64 and ED_F64_NATIVE, FP32 for
 *             ED_F32, complex pairs for ED_C32 / ED_C64. The seeded complex start vector
 *             takes element i = (r_2i, r_2i+1) from the real sequence of ed_start_vector
 *             over 2 dim entries, scaled to unit norm.
 *  schedule   fused H.v kernel variant (1..7 and 14 for ED_F32, 8..13 for ED_F64, 20..23
 *             for ED_C32; 30 (ED_F64) and 31 (ED_F32) are the split-row variants, which
 *             stage a row as two slices of the down states (cut by the occupation of site
 *             0) and run by themselves when the other variants do not fit two rows per SM
 *             in shared memory (or not at all); a variant of another precision or one that
 *             does not fit falls
 *             back to the default one,
 *             see ed_lanczos_schedule); -1 = for bases of at least 2^22 states, the fastest
 *             variant for this basis and dtype, found by timing every variant that fits on
 *             the first run's buffers and remembered by the basis; smaller bases take the
 *             default variant. ED_F64_NATIVE always uses the general kernels.
 *             Batched solves: see ed_lanczos_solve_batched. */
typedef struct {
  int32_t max_steps;
  double tol;
  int32_t reorth;
  uint64_t seed;
  ed_dtype dtype;
  int32_t schedule;
} ed_opts;

#define ED_MAX_STEPS 1000

typedef struct ed_basis ed_basis;
typedef struct ed_lanczos ed_lanczos;

/* ed_build_basis - build both single-species bases and their hop tables on the device.
 * Sec. 2.1 (Eq. 2, Eq. 3): states of each species are unranked from their combinadic rank
 * on the device; for every state and bond with exactly one occupied end, the hop target is
 * ranked and the fermion sign recorded. n_up, n_dn in [0, n_sites]. The basis owns its
 * device tables until ed_basis_destroy. Synchronises `stream`. */
ed_status ed_build_basis(const ed_lattice* lattice, int32_t n_up, int32_t n_dn, void* stream,
                         ed_basis** out);

/* ed_basis_dims - dim_up = C(n_sites, n_up), dim_dn = C(n_sites, n_dn), dim = their product
 * (Eq. 2). Any output pointer may be NULL. */
ed_status ed_basis_dims(const ed_basis* basis, int64_t* dim_up, int64_t* dim_dn, int64_t* dim);

/* ed_basis_filling - the lattice size and particle numbers the basis was built for (Sec. 2.1:
 * L sites, N_up and N_dn fixed). Any output pointer may be NULL. */
ed_status ed_basis_filling(const ed_basis* basis, int32_t* n_sites, int32_t* n_up, int32_t* n_dn);

/* ed_basis_tables - read-only DEVICE views of the basis tables (valid until destroy):
 *  up_bits[dim_up], dn_bits[dim_dn]: uint32 bit strings in rank order.
 *  hop_up[maxhops_up * dim_up], hop_dn[maxhops_dn * dim_dn]: hop k of state r at
 *  [k * dim + r] (column-major ELL, Sec. 2.1 Fig. 2). An entry holds the target rank in
 *  bits 0..29 and the fermion sign in bit 31 (1 = negative). Hops of a state are listed in
 *  bond order; unused slots hold the value dim (an index past the end). */
ed_status ed_basis_tables(const ed_basis* basis, const uint32_t** up_bits,
                          const uint32_t** dn_bits, const int32_t** hop_up,
                          const int32_t** hop_dn, int32_t* maxhops_up, int32_t* maxhops_dn);

void ed_basis_destroy(ed_basis* basis);

/* ed_hv - y = H x (the product of Algorithm 1's first update; Sec. 4 Eqs. 5-6 split it into
 * the up part, which mixes sub-vectors, and the down part, which acts inside each). x and y
 * are DEVICE arrays of dim elements (FP64 for ED_F64 and ED_F64_NATIVE, which both compute
 * in FP64 here; FP32 for ED_F32; complex pairs for ED_C32 / ED_C64), distinct and 16-byte
 * aligned. Asynchronous. */
ed_status ed_hv(const ed_basis* basis, const ed_params* params, ed_dtype dtype, const void* x,
                void* y, void* stream);

/* ed_start_vector - the random unit start vector f_1 of Algorithm 1: element i is
 * 2*u_i - 1 with u_i the top 53 bits of the (i+1)-th SplitMix64 output for `seed`
 * (Steele, Lea & Flood 2014) times 2^-53, then scaled to unit norm in FP64. ED_F32 rounds
 * the normalised FP64 values to nearest. `out` is a DEVICE array of dim elements. */
ed_status ed_start_vector(int64_t dim, uint64_t seed, ed_dtype dtype, void* out, void* stream);

/* ed_start_vector_noalloc - the same start vector as ed_start_vector, computed without
 * allocating any device memory. The paper has no counterpart; this entry point exists for
 * callers that must not allocate device memory while they run, for instance an application
 * whose memory pool already owns the device, or a latency-critical loop that cannot accept
 * the synchronisation a device allocation may cause.
 * Its scratch (the partial sums of the squared norm) is a fixed array of 4096 doubles
 * (32 KB) in the library's static device memory, present on every device that loads the
 * library until the process exits. Sizes needing more partial sums than that are rejected
 * with ED_ERR_ARG (on a GB300, 4 x 152 = 608 are used for any dim). The first call on a
 * device looks up the array's device address with that device current; make that first
 * call before any stream capture. All calls share the array: calls that overlap on the GPU
 * race; consecutive calls on one stream are safe (each call writes every slot it reads).
 * Arguments, layout and errors as ed_start_vector. */
ed_status ed_start_vector_noalloc(int64_t dim, uint64_t seed, ed_dtype dtype, void* out,
                                  void* stream);

/* ed_lanczos_init - allocate a Lanczos state for `basis` with f_1 = f1 (a DEVICE vector of
 * dim elements of opts->dtype, normalised by the library) or, if f1 == NULL, the
 * ed_start_vector of opts->seed. The state owns its work vectors until destroy. */
ed_status ed_lanczos_init(const ed_basis* basis, const ed_opts* opts, const void* f1,
                          void* stream, ed_lanczos** out);

/* ed_lanczos_step - one iteration j of Algorithm 1 with H(params): returns a_j and b_{j+1}
 * (HOST pointers, may be NULL). Returns ED_BREAKDOWN when b_{j+1} vanishes (relative to
 * max_i(|a_i| + b_i), 1e-13); further steps then return ED_ERR_ARG. Synchronises. */
ed_status ed_lanczos_step(ed_lanczos* st, const ed_params* params, double* alpha_j,
                          double* beta_j1);

/* ed_lanczos_run - enqueue nsteps further iterations of Algorithm 1 with H(params) on the
 * state's stream and return without synchronising; steps after a stop (breakdown or
 * max_steps) return at once on the device. If hv_ms is not NULL, CUDA events are recorded
 * on that stream around every fused H.v launch and *hv_ms receives their summed time in
 * milliseconds (this synchronises the stream). */
ed_status ed_lanczos_run(ed_lanczos* st, const ed_params* params, int32_t nsteps, float* hv_ms);

/* ed_lanczos_schedule - the fused H.v variant the state uses (0: the general kernels). */
ed_status ed_lanczos_schedule(const ed_lanczos* st, int32_t* schedule);

/* ed_lanczos_buffers - read-only DEVICE views of the state's two work vectors, for
 * inspection and tests (no counterpart in the paper; Algorithm 1 keeps exactly these two
 * vectors, Sec. 2.2). After step j, *f_next is the buffer of f_{j+1} and *f_cur that of
 * f_j, each an unnormalised vector B with f = scale * B (*scale_next, *scale_cur; for
 * ED_F64 the buffers hold int64 fixed point). Layout: dim_up rows of *ld elements (complex
 * dtypes: pairs), the down rank d at column (*colpos)[d] (*colpos NULL: column d); columns
 * past dim_dn hold 0. Valid until the next call on the state. Any output may be NULL.
 * Synchronises the state's stream. */
ed_status ed_lanczos_buffers(const ed_lanczos* st, const void** f_next, const void** f_cur,
                             double* scale_next, double* scale_cur, int64_t* ld,
                             const int32_t** colpos);

/* ed_lanczos_energy - E0(j) = lowest eigenvalue of T_j (Sec. 2.2), computed on the device
 * by Sturm-sequence bisection to FP64 precision (float-float rounds first, FP64 rounds to
 * finish), and the number of steps j taken. Synchronises. */
ed_status ed_lanczos_energy(ed_lanczos* st, double* E0, int32_t* steps);

void ed_lanczos_destroy(ed_lanczos* st);

/* ed_lanczos_solve - run Algorithm 1 from f1 (as in ed_lanczos_init) until the convergence
 * test of opts passes, b_{j+1} vanishes, or max_steps; returns E0 (HOST) and the steps
 * taken. alpha, beta, E0_hist (HOST, optional, max_steps entries) receive a_1..a_m,
 * b_2..b_{m+1} and E0(1)..E0(m) (the lowest eigenvalue of T_j after every step; without a
 * convergence test (tol = 0) the steps compute E0 only at the stop and the history is
 * computed after the run, all steps in one launch). Returns
 * ED_OK, ED_BREAKDOWN or ED_ERR_NOT_CONVERGED (E0 still set) or an error. Synchronises.
 * The basis keeps the work vectors and the captured CUDA graph of its last solve per
 * (dtype, schedule) for later solves (released by ed_basis_destroy); concurrent solves on one
 * basis from several threads are allowed (the extra ones use private workspaces). */
ed_status ed_lanczos_solve(const ed_basis* basis, const ed_params* params, const ed_opts* opts,
                           const void* f1, void* stream, double* E0, int32_t* steps,
                           double* alpha, double* beta, double* E0_hist);

/* ed_lanczos_solve_mixed - E0 to FP64 accuracy with most steps in FP32. Algorithm 1
 * (Sec. 2.2) runs in FP32 (ED_F32 vectors and H.v) from f1 (an FP32 DEVICE vector of dim
 * elements, or NULL for the seeded start vector of opts->seed) until the convergence test of
 * opts (tol, max_steps) passes, keeping its Lanczos vectors on the device; the Ritz vector
 * psi = sum_j y_j f_j of T_m for its lowest eigenvalue is assembled, and Algorithm 1 runs
 * again in FP64-accurate form (ED_F64) from psi, for at most refine_steps (>= 1) steps with
 * the convergence test |E0(j) - E0(j-1)| <= refine_tol max(|E0(j)|, 1) (refine_tol <= 0:
 * exactly refine_steps steps). Its first step gives a_1 = psi.H psi / psi.psi, the Rayleigh
 * quotient, free of the FP32 rounding of the first phase; the further steps improve on it
 * from a start vector that is already close to the ground state, so the refined run needs
 * few steps, and whatever psi is, its E0 is the FP64-accurate Lanczos value.
 * Outputs (HOST): E0 (the refined run's E0), *steps32 and *E0_fp32 (the FP32 phase's steps
 * and energy), *steps64 (the refined run's steps), *residual = ||H psi - a_1 psi|| / ||psi||
 * (b_2 of the refined run; by the Kato-Temple inequality a_1 - E0_exact <= residual^2 / gap);
 * the four are optional. Returns ED_ERR_NOT_CONVERGED (E0 still set) when the refined run
 * reaches refine_steps with refine_tol > 0. opts->dtype must be ED_F32, opts->reorth 0, the
 * lattice real. The FP32 phase keeps its vectors on the device: it stops after at most as
 * many steps as fit in half the free device memory and in 96 GB, and after at most dim
 * steps. The paper has no mixed-precision form; this is the FP32 variant's route to a
 * 1e-8-accurate E0. Synchronises `stream`. */
ed_status ed_lanczos_solve_mixed(const ed_basis* basis, const ed_params* params,
                                 const ed_opts* opts, const void* f1, int32_t refine_steps,
                                 double refine_tol, void* stream, double* E0, int32_t* steps32,
                                 double* E0_fp32, int32_t* steps64, double* residual);

/* ed_lanczos_solve_batched - Algorithm 1 for n independent instances (basis i with
 * params[i], a HOST array of n) in one persistent cooperative kernel launch, captured in a
 * CUDA graph. opts apply to every instance (dtype ED_F32: FP32 vectors and H.v, dot
 * products as for ED_F32 (compensated FP32 per thread, FP64 across threads); or
 * ED_F64_NATIVE: FP64 vectors and H.v; FP64 a_j, b_j and tridiagonal solve either way;
 * start vector of opts->seed for every instance; reorth 0). The convergence test of opts is evaluated every 4 steps.
 * opts->schedule picks how instances are packed onto groups of CTAs (0..6; 5 sizes groups
 * in proportion to each instance's work per step, 6 to that work times log2 of its
 * dimension, an estimate of its step count); -1 lets the library time every schedule on
 * this batch with the solve itself (at most 200 steps) and keep the fastest (cached per
 * process for the same batch shape). Outputs (HOST arrays of n, steps/status optional):
 * E0[i], steps[i], status[i] (0 running, 1 breakdown, 2 converged, 3 max_steps) and
 * *schedule_used. Returns ED_ERR_NOT_CONVERGED if some instance hit max_steps with tol > 0,
 * ED_ERR_TIMEOUT if a group barrier's bounded wait ran out. Synchronises `stream`. */
ed_status ed_lanczos_solve_batched(int32_t n, const ed_basis* const* bases,
                                   const ed_params* params, const ed_opts* opts, void* stream,
                                   double* E0, int32_t* steps, int32_t* status,
                                   int32_t* schedule_used);

/* ed_lanczos_solve_batched_mixed - E0 of n independent instances to FP64 accuracy with most
 * steps in FP32, in one persistent cooperative kernel launch (the batched form of
 * ed_lanczos_solve_mixed). Per instance: Algorithm 1 (Sec. 2.2) in FP32 as in
 * ed_lanczos_solve_batched (opts: dtype ED_F32, max_steps, tol checked every 4 steps, seed,
 * schedule), keeping its Lanczos vectors on the device (Sum_i dim_i x max_steps x 4 bytes,
 * drawn from a memory pool of the library that keeps the memory reserved in the process for
 * later batched mixed solves; ED_ERR_OOM if it is not available); the eigenvector y of T_m
 * for its lowest eigenvalue by
 * inverse iteration; the Ritz vector psi = sum_j y_j f_j assembled in FP64; then Algorithm 1
 * in FP64 (ED_F64_NATIVE arithmetic) from psi for at most refine_steps (1..ED_MAX_STEPS)
 * steps, with E0 checked every step against refine_tol. Outputs (HOST arrays of n, all but
 * E0 optional): E0[i] of the FP64 phase, steps32[i] and steps64[i] of the two phases,
 * status[i] of the FP64 phase (as in ed_lanczos_solve_batched), *schedule_used. Returns
 * ED_ERR_NOT_CONVERGED if some refinement hit refine_steps with refine_tol > 0,
 * ED_ERR_TIMEOUT if a group barrier's bounded wait ran out. Synchronises `stream`. */
ed_status ed_lanczos_solve_batched_mixed(int32_t n, const ed_basis* const* bases,
                                         const ed_params* params, const ed_opts* opts,
                                         int32_t refine_steps, double refine_tol, void* stream,
                                         double* E0, int32_t* steps32, int32_t* steps64,
                                         int32_t* status, int32_t* schedule_used);

/* ed_lanczos_ground_state - the ground-state vector: Algorithm 1 to convergence (ED_F64
 * only), the eigenvector y of T_m for its lowest eigenvalue (inverse iteration on the
 * device), then the same Lanczos vectors regenerated from f1 and summed, psi = sum_j y_j
 * f_j, exactly in int64 fixed point. psi: DEVICE array of dim FP64, normalised, with the
 * sign fixed so that its largest-magnitude entry (lowest index on ties) is positive. E0 and
 * steps as ed_lanczos_solve. The paper computes E0 only (Sec. 2.2); the vector is the
 * training data of the learned start vector. */
ed_status ed_lanczos_ground_state(const ed_basis* basis, const ed_params* params,
                                  const ed_opts* opts, const void* f1, void* stream, double* psi,
                                  double* E0, int32_t* steps);

/* ed_double_occupancy - double occupancy of a state: D_i = <psi| n_i,up n_i,dn |psi> / <psi|psi>
 * for every site i and D = sum_i D_i. n_i,up n_i,dn is the on-site operator of the
 * interaction term U sum_i n_i,up n_i,dn the paper adds to Eq. 1 (Sec. 1), so for a
 * normalised non-degenerate ground state D = dE0/dU (Hellmann-Feynman). psi: DEVICE array of
 * dim FP64 in the basis order (index rank_up * dim_dn + rank_dn, Sec. 4 Eqs. 5-6), e.g. the
 * output of ed_lanczos_ground_state; any nonzero norm. D_total: HOST double; D_site: HOST
 * array of n_sites doubles or NULL. Accumulated in FP64 in a fixed order (deterministic).
 * ED_ERR_ARG for a NULL or unaligned psi or a zero vector. Synchronises `stream`. */
ed_status ed_double_occupancy(const ed_basis* basis, const double* psi, void* stream,
                              double* D_total, double* D_site);

/* ---------------------------------------------------------------- learned start vector
 * A small network predicts the ground-state amplitude of a basis state from its occupation
 * bits and U; its predictions over the basis are used as f_1 of Algorithm 1 (no counterpart
 * in the paper). Inputs x = (up bits, down bits, U/8) (2L+1 values); two hidden layers of 64
 * tanh units; outputs (a, z); predicted amplitude sign(z) exp(a). Parameters are an FP32
 * master copy, rounded to bfloat16 for every forward pass, FP32 accumulation. Layout (flat):
 * W1 [(2L+1) x 64] input-major, b1 [64], W2 [64 x 64], b2 [64], W3 [64 x 2], b3 [2]. */
typedef struct ed_mlp ed_mlp;

/* ed_mlp_create - network for n_sites-site lattices, Glorot-uniform weights from SplitMix64
 * `seed`, zero biases, zero Adam moments; all work of the handle goes to `stream`. */
ed_status ed_mlp_create(int32_t n_sites, uint64_t seed, void* stream, ed_mlp** out);

/* ed_mlp_params - DEVICE pointer to the FP32 master parameters (read/write) and their count. */
ed_status ed_mlp_params(ed_mlp* mlp, float** params, int64_t* count);

/* ed_mlp_loss_grad - loss of the batch (states idx[n], DEVICE int64 global indices of `basis`;
 * target amplitudes target[n], DEVICE FP64) with per-sample weight weight_scale * target^2:
 *   L = (1/n) sum_k w_k [(a_k - log|t_k|)^2 + log(1 + exp(-sign(t_k) z_k))]  (t_k = 0 skipped)
 * *loss (HOST) and *grad (DEVICE, parameter layout, valid until the next call on the handle)
 * = dL/d(rounded weights). Synchronises the handle's stream when loss != NULL. */
ed_status ed_mlp_loss_grad(ed_mlp* mlp, const ed_basis* basis, double U, const int64_t* idx,
                           const double* target, int64_t n, double weight_scale, double* loss,
                           const float** grad);

/* ed_mlp_train_step - one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on
 * `batch` basis states drawn uniformly (SplitMix64 `seed`) with targets from psi (DEVICE FP64
 * ground-state vector of `basis` at interaction U) and weight_scale = dim. *loss (HOST,
 * optional) = the batch loss before the step. */
ed_status ed_mlp_train_step(ed_mlp* mlp, const ed_basis* basis, double U, const double* psi,
                            int64_t batch, double lr, uint64_t seed, double* loss);

/* ed_mlp_infer - out[i] = predicted amplitude of basis state i at interaction U, for every
 * state of `basis` (DEVICE array of dim, FP32 for ED_F32 else FP64; not normalised). The
 * products run on the tensor cores (bfloat16 operands, FP32 accumulation) and tanh on the
 * special-function unit (relative error about 2^-11); training evaluates tanh exactly to
 * FP32. */
ed_status ed_mlp_infer(ed_mlp* mlp, const ed_basis* basis, double U, ed_dtype dtype, void* out);

void ed_mlp_destroy(ed_mlp* mlp);

/* ed_hv_down_tables - HOST ONLY (no GPU, no CUDA call): the down-hop tables the fused
 * Lanczos H.v builds for one species and one kernel geometry, by the same code the plan
 * uses (the down part of H.v, Sec. 4 Eq. 6; the layout is this library's). For inspection
 * and tests.
 *  hop      [maxhops][dim] int32 (HOST): target rank | sign << 31 (bit 31 set = fermion
 *           sign -1); entries whose rank (bits 0..29) is >= dim are padding.
 *  hop_amp  NULL, or [maxhops][dim] amplitude numbers a, 0 <= 2 a + 1 < 65536 (complex
 *           entries only; NULL = 0).
 *  bits     [dim] uint32 (HOST): bit strings in rank order.
 *  ld       row length: a multiple of 32, at least dim (the library's vectors use dim
 *           rounded up to 32; the split-row tables use longer slices).
 *  V, G     columns per thread (1..8) and shared-memory slots per bank group (8, 16, 32).
 *  complex_entries  0: entries are slots (16-bit in the kernel); 1: slot | signed amplitude
 *           index << 16, index 2 a + s for amplitude number a and sign bit s.
 * Outputs, caller-owned HOST arrays:
 *  table    [rows_cap][ld]: entry of hop step k of column p at table[k ld + p]: the slot
 *           of the target column q, (q & ~(G-1)) | slot_lo[q], or a zero slot ld .. ld+G-1.
 *  rows     the number of table rows (set also when rows_cap is too small).
 *  kpn      [2 ceil(ld / (32 V))]: per chunk of 32 V columns, the rows of +1 hops, then the
 *           rows of -1 hops (complex entries: all hops, then 0).
 *  slot_lo  [ld]: slot of column p within its aligned group of G columns.
 *  colpos   [dim]: column of each down rank (hop count descending, then +1-hop count
 *           descending, then rank).
 * Returns ED_ERR_ARG for inconsistent sizes, rows_cap < rows, an amplitude number out of
 * range, or more than 255 hops of one sign in a column. */
ed_status ed_hv_down_tables(const int32_t* hop, const int32_t* hop_amp, const uint32_t* bits,
                            int64_t dim, int32_t maxhops, int32_t ld, int32_t V, int32_t G,
                            int32_t complex_entries, uint32_t* table, int32_t rows_cap,
                            int32_t* rows, uint8_t* kpn, uint8_t* slot_lo, int32_t* colpos);

/* ed_hv_split_tables - HOST ONLY (no GPU, no CUDA call): the down-hop tables of the split-row
 * fused H.v (schedule 30 / 31) for one species, by the code its plan uses, for inspection and
 * tests. hop [maxhops][dim] and bits [dim] as in ed_hv_down_tables; V columns per thread
 * (1..8); G slots per bank group (8, 16 or 32; the kernels use 16 with V = 2 and 32 with
 * V = 4); site: the site whose occupation cuts the states into slice 0 (occupied) and slice
 * 1 (empty). Slice s holds the columns [cstart[s], cstart[s+1]); its length ld_s is a
 * multiple of 32 V with at least one padding column, and its columns, slot map and in-slice
 * hop rows are those ed_hv_down_tables gives for the slice's own states and in-slice hops
 * (zero slots ld_s .. ld_s + G - 1). Outputs (caller-owned HOST arrays):
 *  table   [rows_cap][cols_cap], row stride *ld: in-slice hop step k of column p at
 *          table[k * ld + p], the slot of the target inside p's slice;
 *  xtable  [rows_cap][cols_cap], row stride *ld: cross-slice hop step k of column p at
 *          xtable[k * ld + p], the target's column inside the other slice (padding: the
 *          other slice's last column, a padding column);
 *  kpn     [4 * (*ld / (32 V))]: per chunk, the in-slice +1 rows, in-slice -1 rows (both in
 *          table), cross +1 rows, cross -1 rows (both in xtable), +1 rows first;
 *  slot_lo [*ld]: slot of column p within its aligned group of G (columns counted from the
 *          slice start); cstart[3] the slice starts (*ld = cstart[2]); colpos [dim] the
 *          column of each down rank; *rows, *xrows the row counts of table and xtable.
 * ED_ERR_ARG when a capacity is too small, a slice does not fit 16 bits, or a column has
 * more than 255 hops of one sign. */
ed_status ed_hv_split_tables(const int32_t* hop, const uint32_t* bits, int64_t dim,
                             int32_t maxhops, int32_t V, int32_t G, int32_t site,
                             uint16_t* table, uint16_t* xtable, int32_t rows_cap,
                             int32_t cols_cap, int32_t* rows, int32_t* xrows, int32_t* ld,
                             int32_t* cstart, uint8_t* kpn, uint8_t* slot_lo, int32_t* colpos);

/* ed_selftest_barrier_timeout - failure-detection self-test of the bounded group barrier
 * used by ed_lanczos_solve_batched: a cooperative launch of `ctas` CTAs (2..64) in which
 * the last CTA never arrives at the barrier; the others must give up after timeout_ms
 * (1..5000) of the GPU's global timer. Returns ED_ERR_TIMEOUT when the bounded wait worked
 * (the context stays usable), ED_OK if the barrier completed, or an error. */
ed_status ed_selftest_barrier_timeout(int32_t ctas, int32_t timeout_ms, void* stream);

/* ed_last_error - message of the last failing call on this thread ("" if none). */
const char* ed_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ED_H_ */
