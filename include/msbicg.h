/*
 * msbicg.h - C ABI of libmsbicg: multi-shifted BiCG for Kramers-Heisenberg
 * (RIXS) response functions on one GB300 (sm_103a).
 *
 * What the library computes (arXiv:2506.09551):
 *   I(w_in, w) = (1/pi) Im <Psi|O1^dag (H - E_G - w - i eta)^{-1} O1|Psi>        (Eq. 1)
 *   |Psi(w_in)> = (H' - E_G - w_in - i Gamma)^{-1} O2 |G>                        (Eq. 2)
 * on a 1D Hubbard chain (Eq. 9) with a core-hole Hamiltonian (Eq. 10), O2 =
 * c^dag_{j,up}, O1 = c_{j,up}.  All |Psi(w_in)> come from one seed Krylov
 * recurrence shared by every incident energy (Eqs. 4-8, App. C, Alg. 1); the
 * second step is a Lanczos continued fraction for every w_in.
 *
 * Conventions for every call
 *   - Vectors are caller-owned DEVICE buffers unless stated otherwise.
 *     Complex vectors are interleaved (re, im): 16 bytes per element for
 *     MSB_FP64, 8 bytes for MSB_FP32_MIXED.  A block of nvec vectors is stored
 *     vector after vector (vector k starts at element k * dim).
 *   - Basis order: a many-body state (u, d) of the (n_up, n_dn) sector has
 *     index rank(u) * D_dn + rank(d); rank is the position of the L-bit
 *     occupation string among all strings of that popcount in ascending order
 *     (bit i = site i).  Fermionic signs use the Jordan-Wigner order "all up
 *     orbitals (site 0..L-1), then all down orbitals".
 *   - Handles (msb_basis, msb_op) are library-owned: create/destroy pairs.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is ordered on it.  Calls that return host results
 *     synchronise the stream before returning.
 *   - No exceptions cross the ABI: every call returns msb_status and, on
 *     failure, sets a thread-local message readable with msb_last_error().
 *   - There is no CPU fallback: without a usable CUDA device every compute
 *     call returns MSB_ECUDA.
 */
#ifndef MSBICG_H
#define MSBICG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MSB_OK = 0,
    MSB_EINVAL = 1,       /* invalid argument (sizes, pointers, model)            */
    MSB_ENOMEM = 2,       /* device or pinned-host allocation failed              */
    MSB_ECUDA = 3,        /* CUDA runtime error, or no usable device               */
    MSB_EBREAKDOWN = 4,   /* (p, A p) = 0, zeta_{m+1} = 0, or (r, r) = 0 with r != 0 */
    MSB_EMAXITER = 5,     /* iteration cap reached; partial results are written    */
    MSB_ENONFINITE = 6,   /* NaN or Inf met in a recurrence scalar                 */
    MSB_ETIMEOUT = 7      /* reserved: a bounded device wait ran out               */
} msb_status;

typedef enum {
    MSB_FP64 = 0,         /* complex double vectors, FP64 apply and updates         */
    MSB_FP32_MIXED = 1    /* complex float vectors and apply; FP64 dots, zeta/alpha/
                             beta recurrences, ground state and continued fraction */
} msb_precision;

typedef struct { double re, im; } msb_complex;

/* Hubbard cluster and RIXS transition (Eqs. 9-10; Sec. III).
 * H' = H - Uc (n_{j,up} + n_{j,dn}) on the sector with the O2 electron added:
 * the core hole sits on the site j = core_site where O2 = c^dag_{j,o2_spin}
 * acted, and the edge energy E_edge is absorbed into w_in.  O1 = c_{j,o1_spin}
 * fills the core hole; o1_spin == o2_spin is the spin-conserving channel (final
 * states in the ground sector), o1_spin != o2_spin the spin-flip channel (final
 * states with one o1_spin electron fewer and one o2_spin electron more).  A
 * zero-initialised tail (o2_spin = o1_spin = lx = 0, tp = 0) is the up-spin
 * channel on a chain. */
typedef struct {
    int L;            /* sites, 3 <= L <= 16 for a ring, 2 <= L <= 16 open       */
    int n_up, n_dn;   /* electrons of the ground-state sector                    */
    int periodic;     /* chain: 1 ring, 0 open (ignored for a 2D cluster)        */
    double t;         /* nearest-neighbour hopping (Eq. 9)                       */
    double U;         /* on-site repulsion (Eq. 9)                               */
    double Uc;        /* core-hole potential (Eq. 10)                            */
    int core_site;    /* j of O2 = c^dag_{j,o2_spin}, O1 = c_{j,o1_spin}          */
    int o2_spin;      /* 0 = up, 1 = down                                        */
    int o1_spin;      /* 0 = up, 1 = down                                        */
    int lx;           /* 0: chain of L sites; > 0: periodic lx x (L / lx) cluster,
                         site x + lx y, lx >= 3 and L / lx >= 3                  */
    double tp;        /* diagonal (next-nearest-neighbour) hopping t' of a 2D
                         cluster; bonds (x,y)-(x+1,y+1) and (x,y)-(x-1,y+1)      */
    double flux;      /* magnetic flux through a ring (Peierls phases): the hop of
                         an electron from site i to i + 1 carries exp(i flux / L),
                         the reverse hop exp(-i flux / L).  Nonzero makes H
                         complex Hermitian: only the dual solver
                         (msb_multishift_bicg_dual_solve) and msb_op_apply take
                         such an operator.  Chain only (lx = 0).                 */
} msb_model;

/* Parameters of the whole map (Eqs. 1-2). */
typedef struct {
    double Gamma;        /* inverse core-hole lifetime (Eq. 2), > 0             */
    double eta;          /* broadening replacing i0+ in Eq. 1, > 0              */
    double gs_tol;       /* ground state: ||H G - E_G G|| <= gs_tol max(1,|E_G|) */
    int gs_maxit;        /* Lanczos steps per restart for the ground state       */
    double solve_tol;    /* per shift: ||r^(w)|| <= solve_tol ||O2 G||            */
    int maxit;           /* seed iteration cap                                   */
    double cf_tol;       /* continued fraction: stop when no I(w) of a row moves
                            by more than cf_tol * max_w |I| over cf_check levels */
    int cf_check;        /* levels between convergence checks (e.g. 50)          */
    int cf_maxdepth;     /* depth cap of the continued fraction                  */
    int seed_index;      /* incident energy used as the seed; -1: nearest to 0   */
    int block;           /* lag of the fused per-shift update (1..16; 0 = auto)  */
    msb_precision precision;
} msb_map_params;

/* Counters and timings filled by the solve and map calls (any field may be 0). */
typedef struct {
    int iterations;             /* seed iterations = MVMs of the shared recurrence    */
    int n_converged;            /* shifts that met the tolerance                      */
    int64_t matvecs;            /* all operator applications (ground state, solve, CF) */
    int64_t flushes;            /* launches of the fused per-shift update             */
    double seed_residual;       /* ||r_m|| / ||b|| of the seed at exit                */
    double max_shift_residual;  /* max over shifts of ||r_m|| / (|zeta_m| ||b||)      */
    double E_G;                 /* ground-state energy used                           */
    double gs_residual;         /* ||H G - E_G G|| of the ground state                 */
    int cf_depth_max;           /* deepest continued fraction used                    */
    int cf_depth_min;
    double seconds_ground_state, seconds_solve, seconds_second_step, seconds_total;
    int64_t device_bytes;       /* workspace bytes allocated by the call              */
    int64_t kernel_launches;    /* kernels launched by the call                       */
} msb_solve_info;

typedef struct msb_basis msb_basis;
typedef struct msb_op msb_op;

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                               */
/* ------------------------------------------------------------------------ */

/* Message of the last failed call on this thread ("" if none).  The pointer
 * stays valid until the next failing call on the same thread. */
const char *msb_last_error(void);

/* Library version string, e.g. "msbicg 0.1 sm_103a". */
const char *msb_version(void);

/* Fill `p` with the defaults used by the map workloads: Gamma 0.3, eta 0.1,
 * gs_tol 1e-12, gs_maxit 300, solve_tol 1e-10, maxit 5000, cf_tol 1e-10,
 * cf_check 50, cf_maxdepth 4000, seed_index -1, block 0, MSB_FP64. */
void msb_map_params_default(msb_map_params *p);

/* ------------------------------------------------------------------------ */
/* Sector basis (host)                                                       */
/* ------------------------------------------------------------------------ */

/* Occupation-number basis of the (n_up, n_dn) sector of an L-site chain: the
 * Hilbert space of Eq. (A1) in the paper's notation.  Host-only object.
 * Errors: MSB_EINVAL if L is outside 1..16 or n outside 0..L. */
msb_status msb_basis_create(int L, int n_up, int n_dn, msb_basis **out);

/* Sizes: D_up = C(L, n_up), D_dn = C(L, n_dn), dim = D_up * D_dn (any output may be NULL). */
msb_status msb_basis_dims(const msb_basis *b, int64_t *D_up, int64_t *D_dn, int64_t *dim);

/* Copy the occupation strings of one spin species (0 = up, 1 = down) in rank
 * order into the HOST array `out` (D_species entries). */
msb_status msb_basis_states(const msb_basis *b, int species, uint32_t *out);

void msb_basis_destroy(msb_basis *b);

/* Row order of the continued fraction (second step of Eq. 1).  That step needs
 * only the Lanczos coefficients, so its internal vectors may hold each row's
 * down-spin states in any fixed order.  The row-tiled apply kernels run their
 * down-spin loop to the largest hop count among a warp's elements, so position
 * p of a row holds down state order[p], the states sorted by their number of
 * down-spin hops (descending, ties in rank order).  No effect on any result.
 * Host only, no device.  order: HOST array of D_dn entries (a permutation of
 * 0..D_dn-1).  Errors: MSB_EINVAL if D_dn is not below 32768, or periodic with
 * L < 3. */
msb_status msb_basis_row_order(const msb_basis *b, int periodic, uint16_t *order);

/* Shared-memory placement and hop schedule of a down-spin row used by the FP32
 * continued-fraction apply.  That kernel stages each row of a vector in shared
 * memory (in the row order above) and gathers the down-spin hop targets from
 * it, one hop per position per round, for the largest hop count of the warp's
 * positions.  Since the hop table is the same for every row, the library
 * chooses once per sector (deterministic searches; no effect on any result
 * beyond the order of a sum) the slot of each position and the round of each
 * of its hops, so that the gathers of a half-warp hit fewer shared-memory bank
 * conflicts.  Host only, no device.
 * slot: HOST array of D_dn entries (may be NULL): slot[p] for each position p
 * (a permutation of 0..D_dn-1).  width (may be NULL): the table width W, the
 * number of bonds (L for a ring, L - 1 for an open chain).  hops: HOST array of
 * W x D_dn entries (may be NULL): hops[k * D_dn + p] = (target position << 1 |
 * sign bit) read by position p in round k, or D_dn << 1 for an idle round (the
 * zero word); every hop of p appears once in rounds below its warp's largest
 * hop count.  cost_plain / cost_layout (may be NULL): the mean worst-bank
 * count per half-warp gather for slot[p] = p with the hops in table order, and
 * for the chosen slots and rounds (1 is conflict free).  Errors: MSB_EINVAL if
 * D_dn is odd or not below 32768, or periodic with L < 3. */
msb_status msb_basis_row_layout(const msb_basis *b, int periodic, uint16_t *slot, int *width, uint16_t *hops,
                                double *cost_plain, double *cost_layout);

/* ------------------------------------------------------------------------ */
/* Operators A = H, H' (matrix-free) or a user CSR matrix                    */
/* ------------------------------------------------------------------------ */

/* Matrix-free Hubbard operator (Eq. 9 on the model's chain or 2D cluster).
 * sector = 0: H on the ground sector (n_up, n_dn); 1: H' of Eq. (10) on the
 * intermediate sector, the ground sector plus the O2 electron (o2_spin), with
 * the core hole on core_site; 2: H on the final sector, the intermediate
 * sector minus the O1 electron (o1_spin) -- the ground sector again unless the
 * channel flips the spin.  The hopping tables are built on the host and copied
 * to the current device.
 * Errors: MSB_EINVAL (model or sector out of range), MSB_ECUDA, MSB_ENOMEM. */
msb_status msb_op_create_hubbard(const msb_model *model, int sector, msb_op **out);

/* General real symmetric sparse matrix in CSR form (HOST arrays: rowptr[n+1],
 * col[nnz], val[nnz]); copied to the device.  Symmetry is assumed, not checked;
 * the solver needs A^T = A (App. A).  Columns must lie in [0, n). */
msb_status msb_op_create_csr(int64_t n, const int64_t *rowptr, const int32_t *col,
                             const double *val, msb_op **out);

/* Direct sum (block-diagonal operator) of n <= 16 Hubbard operators ops[i]
 * (from msb_op_create_hubbard), each with a real diagonal shift shifts[i]
 * (HOST array, NULL = all zero): A = (H_0 + s_0) (+) (H_1 + s_1) (+) ...
 * Vectors of A are the parts' vectors one after another (part 0 first).  One
 * launch of msb_op_apply or of the solver's MVM covers every part, so one
 * multi-shift solve (Alg. 1) serves independent clusters of uneven size: with
 * s_i = -E_G of cluster i, the seed system (A - w_seed - i Gamma) has the
 * cluster's own E_G in every block and the shifts w_in - w_seed are common.
 * The parts are NOT owned: they must outlive the sum.  msb_ground_state and
 * msb_continued_fraction reject a direct sum (MSB_EINVAL).
 * Errors: MSB_EINVAL (n outside 1..16, a part that is not a Hubbard operator or
 * lives on another device, a non-finite shift). */
msb_status msb_op_create_direct_sum(const msb_op *const *ops, const double *shifts, int n, msb_op **out);

msb_status msb_op_dim(const msb_op *op, int64_t *dim);

void msb_op_destroy(msb_op *op);

/* y_k = (A + c0 I) x_k for k < nvec (the MVM of Alg. 1).  x and y are device
 * blocks of nvec complex vectors (FP64 or FP32 by `prec`); x and y must not
 * overlap.  Asynchronous on `stream`. */
msb_status msb_op_apply(msb_op *op, msb_complex c0, const void *x, void *y, int nvec,
                        msb_precision prec, void *stream);

/* ------------------------------------------------------------------------ */
/* Transition operators between sectors (Eqs. 1-2 with the dipole operators  */
/* reduced to a single orbital)                                              */
/* ------------------------------------------------------------------------ */

/* y_k = c^dag_{site,up} x_k: x in the (n_up, n_dn) sector of `model`, y in
 * (n_up + 1, n_dn).  Complex vectors per `prec`; asynchronous. */
msb_status msb_apply_cdag_up(const msb_model *model, int site, const void *x, void *y,
                             int nvec, msb_precision prec, void *stream);

/* y_k = c_{site,up} x_k: x in (n_up + 1, n_dn), y in (n_up, n_dn). */
msb_status msb_apply_c_up(const msb_model *model, int site, const void *x, void *y,
                          int nvec, msb_precision prec, void *stream);

/* ------------------------------------------------------------------------ */
/* Ground state (Sec. III: |G>, E_G; Lanczos in FP64 in every mode)         */
/* ------------------------------------------------------------------------ */

/* Lowest eigenpair of the real symmetric operator H by Lanczos, restarted from
 * its Ritz vector until ||H g - E g|| <= tol * max(1, |E|).  `start` is an
 * optional device real vector (NULL: a counter-based pseudo-random vector);
 * `g` is a device real double vector of length dim (caller-owned, output,
 * unit norm).  E_G and residual are host outputs.  Synchronises `stream`.
 * Errors: MSB_EMAXITER if 20 restarts do not reach tol (g, E_G still written);
 * MSB_EINVAL for a direct sum (msb_op_create_direct_sum: take each part's). */
msb_status msb_ground_state(msb_op *H, double tol, int maxit, const double *start,
                            double *E_G, double *g, double *residual, void *stream);

/* The same ground state for callers that cannot allocate device memory: a
 * process whose device memory is owned by another allocator under a fixed
 * budget (a framework's caching pool, a server that reserved its memory at
 * start-up), where one more cudaMalloc fails or fragments that budget.
 * The paper has no counterpart: this is a deployment variant.  It allocates
 * nothing: its scratch is a fixed array inside the library image of
 * 5 * 2^20 doubles plus a few KB (about 42 MB), held on every GPU that loads
 * the library until the process exits.  Limits: dim <= 1048576 (2^20) and
 * maxit <= 1024, else MSB_EINVAL.  The array's device address is looked up at
 * the start of every call, on the caller's current device.  Work is ordered on
 * `stream` itself; the call synchronises `stream` and copies the Lanczos
 * coefficients to the host at every step, and returns after a final
 * synchronisation.  All calls share the array and it keeps the previous
 * call's contents (every part a call reads is written first in that call):
 * calls that overlap on the GPU race.  Arguments and results as
 * msb_ground_state. */
msb_status msb_ground_state_noalloc(msb_op *H, double tol, int maxit, const double *start,
                                    double *E_G, double *g, double *residual, void *stream);

/* ------------------------------------------------------------------------ */
/* Multi-shifted BiCG (App. C; Alg. 1 in corrected form)                     */
/* ------------------------------------------------------------------------ */

/* Solve (A + c0 I - s_k I) x_k = b for every shift s_k (HOST array, n_shifts
 * <= 4096) from one seed recurrence on A + c0 I, which must be complex
 * symmetric (real symmetric A; c0 complex).  b: device complex vector; x:
 * device block of n_shifts complex vectors (caller-owned, output).  A shift is
 * frozen once ||r_m|| / |zeta_m^(k)| <= tol ||b||.  Optional HOST outputs
 * (may be NULL): iters[k], resid[k] (that ratio / ||b|| at freeze), converged[k].
 * `block` (1..16, 0 = auto) lags the fused per-shift update: the vectors
 * p^(k), x^(k) are advanced once every `block` iterations from the stored seed
 * residuals, with coefficients from the same recurrences.
 * Returns MSB_EMAXITER (results still written) if a shift did not converge
 * within maxit, MSB_EBREAKDOWN / MSB_ENONFINITE on a failed recurrence,
 * MSB_EINVAL for an operator with Peierls phases (not complex symmetric: use
 * msb_multishift_bicg_dual_solve). */
msb_status msb_multishift_bicg_solve(msb_op *A, msb_complex c0, const void *b,
                                     const msb_complex *shifts, int n_shifts, double tol,
                                     int maxit, int block, msb_precision prec, void *x,
                                     int *iters, double *resid, int *converged,
                                     msb_solve_info *info, void *stream);

/* The same multi-shift solve for an operator A that is Hermitian but not real
 * symmetric (a Hubbard ring with Peierls phases, msb_model.flux != 0), where
 * A + c0 is not complex symmetric and the bilinear form no longer makes the
 * residuals biorthogonal.  Dual-space BiCG (App. A): a second recurrence in the
 * space of (A + c0)^dagger = A + conj(c0), with dual residual r~ (r~_0 = b) and
 * direction p~, and Hermitian products: alpha = <r~|r> / <p~|A p>,
 * r~ <- r~ - conj(alpha) (A + conj(c0)) p~, p~ <- r~ + conj(beta) p~.  Two operator
 * applications per iteration (info->matvecs = 2 * iterations).  The shifted
 * residuals stay collinear with the seed's (App. B), so the per-shift zeta /
 * alpha / beta recurrences and the fused per-shift update are those of
 * msb_multishift_bicg_solve.  Arguments, outputs and errors as that call; it
 * also accepts a real symmetric A (then it converges to the same solutions). */
msb_status msb_multishift_bicg_dual_solve(msb_op *A, msb_complex c0, const void *b,
                                          const msb_complex *shifts, int n_shifts, double tol,
                                          int maxit, int block, msb_precision prec, void *x,
                                          int *iters, double *resid, int *converged,
                                          msb_solve_info *info, void *stream);

/* Adaptive reseeding (App. E, Fig. 5) around the solve above.  Solves
 * (A + c0 I - s_k I) x_k = b for every shift, first from the seed system
 * A + c0 - s_{seed_index}.  After each run, every solved shift's true residual
 * b - (A + c0 - s_k) x_k (one operator application per shift) is compared with
 * the recursive residual r_m / zeta_m^k the recurrence carried (Eq. 4):
 * dr[k] = ||true - recursive||.  A shift is accepted when it converged and
 * dr[k] <= reseed_tol ||b||.  The rejected shift closest to the current seed
 * becomes the next seed and the rejected shifts are solved again from it;
 * accepted shifts keep their solutions.  Stops when all are accepted or after
 * max_seeds seeds.  x: device block of n_shifts vectors (output).  HOST
 * outputs (may be NULL): converged[k], accepted[k], dr[k] (of the last run that
 * solved shift k), seeds[max_seeds] (the seed indices used, in order) and
 * *n_seeds.  info->iterations and ->matvecs sum over the runs.  Returns
 * MSB_EMAXITER (results written) if some shift is not accepted, MSB_ENONFINITE
 * on a failed recurrence.  Allocates two n_shifts x dim work blocks. */
msb_status msb_multishift_bicg_reseeded(msb_op *A, msb_complex c0, const void *b, const msb_complex *shifts,
                                        int n_shifts, double tol, int maxit, int block, msb_precision prec,
                                        double reseed_tol, int seed_index, int max_seeds, void *x, int *converged,
                                        int *accepted, double *dr, int *seeds, int *n_seeds, msb_solve_info *info,
                                        void *stream);

/* The paper's baseline for Eq. 2 (Sec. III, Fig. 4): every shift solved on its
 * own by BiCGStab (van der Vorst 1992; x_0 = 0, shadow residual b, Hermitian
 * products), (A + c0 I - s_k I) x_k = b until ||r_k|| <= tol ||b||.  All shifts
 * advance together (each launch covers every active shift) but each has its own
 * Krylov space: two operator applications per iteration per shift, against one
 * per iteration for all shifts in msb_multishift_bicg_solve.  b: device vector;
 * x: device block of n_shifts vectors (output).  HOST outputs (may be NULL):
 * iters[k], resid[k] (recursive ||r_k|| / ||b||), converged[k], restarts[k].
 * A shift whose recurrence breaks down (<r^|v> or <r^|r> vanishing, omega = 0,
 * a non-finite scalar) restarts from its current iterate with r = r^ = b - A_k x
 * (one more product), at most 64 times.
 * info->matvecs = 2 * sum_k iters[k] + sum_k restarts[k];
 * info->iterations = max_k iters[k].
 * Allocates four n_shifts x dim work blocks.  Returns MSB_EMAXITER (results
 * written) if a shift did not converge within maxit or broke down. */
msb_status msb_bicgstab_solve(msb_op *A, msb_complex c0, const void *b, const msb_complex *shifts, int n_shifts,
                              double tol, int maxit, msb_precision prec, void *x, int *iters, double *resid,
                              int *converged, int *restarts, msb_solve_info *info, void *stream);

/* ------------------------------------------------------------------------ */
/* Second step: batched Lanczos continued fraction (Eq. 1; Sec. III)         */
/* ------------------------------------------------------------------------ */

/* For each of n_vec device complex vectors phi_k (block, per `prec`) of the
 * space of the real symmetric operator H, compute
 *   I[k][i] = (1/pi) Im <phi_k|(H - E0 - w_i - i eta)^{-1}|phi_k>
 * by a Hermitian Lanczos continued fraction of converged depth (see
 * msb_map_params.cf_tol / cf_check / cf_maxdepth).  I_out is a HOST array
 * n_vec x n_w; depth (HOST, nullable) receives each row's depth.
 * The input vectors are not modified.  Synchronises `stream`.
 * Errors: MSB_EINVAL for bad sizes or a direct sum (its columns would mix the
 * parts; msb_rixs_map_clusters runs one fraction over several clusters). */
msb_status msb_continued_fraction(msb_op *H, const void *phi, int n_vec, double E0,
                                  const double *w, int n_w, double eta, double cf_tol,
                                  int cf_check, int cf_maxdepth, msb_precision prec,
                                  double *I_out, int *depth, void *stream);

/* ------------------------------------------------------------------------ */
/* The whole RIXS map (Eqs. 1-2)                                             */
/* ------------------------------------------------------------------------ */

/* I_out[k][i] = I(w_in[k], w[i]) for the model, HOST arrays w_in[n_in], w[n_w]
 * and HOST output I_out[n_in * n_w].  G: optional device real unit vector of
 * the ground sector with energy E_G (NULL: computed by msb_ground_state with
 * params->gs_tol).  The seed system is w_in[seed_index]; the shifts are
 * w_in[k] - w_in[seed].  Synchronises `stream`; all workspace is allocated
 * and freed inside the call.  Returns MSB_EMAXITER if some w_in did not
 * converge (the map is still written). */
msb_status msb_rixs_map(const msb_model *model, const msb_map_params *params,
                        const double *G, double E_G, const double *w_in, int n_in,
                        const double *w, int n_w, double *I_out, msb_solve_info *info,
                        void *stream);

/* ------------------------------------------------------------------------ */
/* Autotuner                                                                 */
/* ------------------------------------------------------------------------ */

/* Timed trials, on the operators of `model`, of the launch choices that leave
 * the results unchanged up to the rounding order of a block reduction: the lag
 * B in {1, 2, 4, 8, 16} of the fused per-shift update of a solve with n_in
 * shifts (FP32 or FP64 per `prec`), and the shape of the row-tiled
 * continued-fraction apply: threads per CTA (128 or 256) for MSB_FP64; for
 * MSB_FP32_MIXED 1 (one column per CTA, 6 CTAs per SM), 2 (two columns per CTA),
 * 3 (one column, 8 CTAs per SM) or 4 (one column per 512-thread CTA, 4 CTAs per
 * SM), returned in *cf_threads.  Each candidate is
 * timed with CUDA events as the difference of a 2K- and a K-iteration run (the
 * allocations of a call cancel); an apply shape is taken only if its
 * 32-level continued fraction agrees with the first shape's (relative L2 1e-10
 * in FP64, 1e-4 in FP32), and the fixed default shape is kept unless another is
 * at least 2% faster.  The fastest choices are cached for the whole
 * process, keyed by the problem's shape (intermediate dimension, n_in and
 * precision for B; row length, row count and precision for the threads), and
 * used by every later call that leaves them automatic (params->block or the
 * solver's `block` = 0).  HOST outputs (may be NULL): the choices, and the
 * measured milliseconds per iteration for each B (5 values) and per level for
 * each apply shape (4 values; the last two are 0 for FP64).  Allocates and frees its own work
 * vectors; synchronises `stream`.  The paper has no counterpart. */
msb_status msb_autotune(const msb_model *model, msb_precision prec, int n_in, int *block, int *cf_threads,
                        double *block_ms, double *cf_ms, void *stream);

/* Forget every cached autotuned choice (later calls use the fixed defaults). */
void msb_autotune_forget(void);

/* ------------------------------------------------------------------------ */
/* Kernel profiling                                                          */
/* ------------------------------------------------------------------------ */

/* Per kernel class: launches, summed CUDA-event durations (each launch is
 * bracketed by events on the stream it runs on), and the algorithmic DRAM
 * bytes and floating-point operations of those launches (what the method
 * must move / compute for the sizes involved: each vector read or written
 * once per use, hop tables and scalars not counted). */
typedef struct {
    char name[48];
    int64_t launches;
    double ms;
    double alg_bytes;
    double alg_flops;
} msb_kernel_stat;

/* Turn profiling on or off for the whole process.  While on, the solver
 * launches its kernels directly instead of replaying CUDA graphs, so every
 * launch can be timed; the arithmetic is unchanged. */
void msb_profile_enable(int on);

/* Forget all collected statistics. */
void msb_profile_reset(void);

/* Copy up to `max` kernel classes with at least one launch into `out` (HOST
 * array; may be NULL to count) and return how many there are. */
int msb_profile_read(msb_kernel_stat *out, int max);

/* Maps for several right-hand sides of one model: O2 = c^dag_{j,up}, O1 =
 * c_{j,up} and the core hole on site j for every j in sites[n_sites] (Eqs. 1-2
 * per site; the batched workload of one cluster with one right-hand side per
 * core site).  One ground state; ONE multi-shift solve on the direct sum of the
 * sites' (H'_j - E_G) for the concatenated right-hand side (O2_j |G>)_j (every
 * launch of the solve covers all sites); one continued fraction over all
 * n_sites * n_in columns, which share H.  model->core_site is ignored.  I_out:
 * HOST array n_sites x n_in x n_w (site slowest).  Requires n_sites <= 16 and
 * n_sites * n_in <= 65535.  Synchronises `stream`. */
msb_status msb_rixs_map_sites(const msb_model *model, const msb_map_params *params, const int *sites,
                              int n_sites, const double *w_in, int n_in, const double *w, int n_w,
                              double *I_out, msb_solve_info *info, void *stream);

/* Maps of several independent clusters, models[n_clusters] (n_clusters <= 16;
 * any L, fillings, boundary and core site each), computed together: one FP64
 * ground state per cluster, then ONE multi-shift solve on the direct sum of
 * the clusters' (H'_c - E_G,c) for the concatenated right-hand side
 * (O2|G_c>)_c (every kernel launch of the solve covers all clusters), then ONE
 * continued fraction over all n_clusters * n_in columns, each column applying
 * its own cluster's H (Eqs. 1-2 per cluster).  The solve tolerance is applied
 * per cluster: the joint residual bound is tol * min_c ||O2 G_c||.
 * I_out: HOST array n_clusters x n_in x n_w (cluster slowest); E_G_out: HOST
 * array n_clusters, or NULL.  Requires n_clusters * n_in <= 65535.
 * Synchronises `stream`.  Errors as msb_rixs_map. */
msb_status msb_rixs_map_clusters(const msb_model *models, int n_clusters, const msb_map_params *params,
                                 const double *w_in, int n_in, const double *w, int n_w, double *I_out,
                                 double *E_G_out, msb_solve_info *info, void *stream);

/* Momentum-resolved maps (the coherent sum over core sites, Sec. III): for every
 * site j the map of msb_rixs_map_sites is formed up to phi_j = c_{j,up} Psi_j
 * (one ground state; one multi-shift solve over all sites' H'), then
 *   phi_q = sum_j exp(i q j) phi_j   and
 *   I_q(w_in, w) = (1/pi) Im <phi_q|(H - E_G - w - i eta)^{-1}|phi_q>
 * by one continued fraction over all n_q * n_in columns.  qs: HOST array of
 * n_q momenta (radians per site; over q = 2 pi k / L the maps sum to L times the
 * sum of the single-site maps).  model->core_site is ignored.  I_out: HOST array
 * n_q x n_in x n_w (q slowest).  Requires n_q * n_in <= 65535 and
 * L * n_in <= 65535 (L <= 16).  Synchronises `stream`.  Errors as msb_rixs_map. */
msb_status msb_rixs_map_q(const msb_model *model, const msb_map_params *params, const double *qs, int n_q,
                          const double *w_in, int n_in, const double *w, int n_w, double *I_out,
                          msb_solve_info *info, void *stream);

/* Same map with the operators already built and the result left on the
 * device: H = msb_op_create_hubbard(model, 0), Hp = msb_op_create_hubbard(model,
 * 1) of one model (checked); w_in, w are HOST grids (copied in); I_dev is a
 * DEVICE output of n_in * n_w doubles.  For repeated maps of one model, and to
 * time the path with its inputs resident in device memory.
 * Synchronises `stream`. */
msb_status msb_rixs_map_ops(msb_op *H, msb_op *Hp, const msb_map_params *params, const double *G,
                            double E_G, const double *w_in, int n_in, const double *w, int n_w,
                            double *I_dev, msb_solve_info *info, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MSBICG_H */
