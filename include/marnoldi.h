/*
 * marnoldi.h -- C ABI of libmarnoldi, the GB300 (sm_103a) multiple Arnoldi solver.
 *
 * The library implements the data-parallel hot path of the multiple Arnoldi
 * (mArnoldi) method of Hoshi, Yamazaki and Akiyama (arXiv:1307.3218, Section 2):
 * for every requested basis index j of a sparse real-symmetric LCAO pair (H, S),
 * S positive definite, it
 *   1. builds the nu-dimensional Krylov subspace L_nu^(j) that contains e_j
 *      (span{e_j, H e_j, ..., H^(nu-1) e_j}) with an S-orthonormal basis K
 *      (Gram-Schmidt in the S inner product against the exact S-Gram matrix
 *      of the stored vectors);
 *   2. solves the nu x nu standard subspace eigenproblem H_sub = K^T H K
 *      (levels eps_a, vectors v_a);
 *   3. turns the subspace eigenpairs into the columns of the Green's function
 *      (z S - H)^-1 e_j (Eq. 1), of the density matrix and of the
 *      energy-density matrix, and into the band energy, at a Fermi level mu
 *      found by bisection on the electron count (or given).
 *
 * Conventions
 *   - Matrices are BSR with 4x4 blocks: row_ptr[n_block_rows + 1] (int64,
 *     row_ptr[0] = 0), col_idx[nnzb] (int32, strictly ascending inside a block
 *     row, the diagonal block present), vals[nnzb][4][4] row-major doubles.
 *     Orbital index of (atom I, orbital a) is 4 I + a; M = 4 n_block_rows.
 *     H and S share one pattern, which must be symmetric.
 *   - Outputs on H's pattern use the same BSR layout: entry [k][a][b] of block
 *     k = (I, J) is row 4 I + a, column 4 J + b.  Column 4 J + b of rho,
 *     rho^E and G(z) is produced by the subspace of j = 4 J + b; the columns
 *     are not symmetrised.
 *   - Energies in the units of H (eV for the bundled models); kT in the same
 *     units; f(x) = 1 / (1 + e^x), spin factor 2.
 *   - Every function returns a marnoldi_status; nothing throws or exits
 *     across the ABI.  On failure marnoldi_last_error(ctx) describes it.
 *   - Host pointers unless a name ends in _device.  The caller owns every
 *     array it passes; the library copies what it keeps.
 *   - One context per structure.  A context's calls are issued on its CUDA
 *     stream and are not thread-safe; different contexts are independent and
 *     may be used from different threads at the same time.
 */
#ifndef MARNOLDI_H
#define MARNOLDI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct marnoldi_ctx marnoldi_ctx;

typedef enum {
    MARNOLDI_OK = 0,
    MARNOLDI_EINVAL = -1,    /* bad argument or malformed matrices */
    MARNOLDI_ENOTSPD = -2,   /* S shown not positive definite */
    MARNOLDI_ENOMEM = -3,    /* device or host allocation failed */
    MARNOLDI_ECUDA = -4,     /* a CUDA call failed */
    MARNOLDI_ETIMEOUT = -5,  /* a bounded device loop ran out of iterations */
    MARNOLDI_ESTATE = -6,    /* call out of order (e.g. density before solve) */
    MARNOLDI_ENOCONV = -7,   /* the subspace eigensolver or the bisection did not converge */
    MARNOLDI_EPENDING = -8   /* a server request has not finished within the wait's timeout */
} marnoldi_status;

typedef enum {
    MARNOLDI_FP64 = 0,   /* every step in FP64 */
    MARNOLDI_MIXED = 1   /* FP32 SpMM and Krylov-vector storage; FP64 inner products,
                            Gram-Schmidt coefficients, eigensolve and accumulation */
} marnoldi_precision;

/* Device allocator hook: alloc(bytes, stream, user) returns device memory usable
 * in the order of `stream`; free(ptr, bytes, stream, user) releases it.  Passing
 * NULL for both restores the default (cudaMallocAsync / cudaFreeAsync).
 * Process-wide; set it before creating contexts.  Returns MARNOLDI_OK. */
typedef void *(*marnoldi_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*marnoldi_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
int marnoldi_set_allocator(marnoldi_alloc_fn alloc, marnoldi_free_fn free_fn, void *user);

/*
 * Validate and upload one structure (H, S) to the device (arXiv:1307.3218,
 * Section 2: sparse real-symmetric M x M LCAO matrices, S positive definite).
 *
 *   out           receives a new context (NULL on failure).
 *   n_block_rows  number of atoms (>= 1).
 *   row_ptr, col_idx, H_vals, S_vals   the BSR pair described above (host).
 *   orbital_mask  n_block_rows*4 bytes, 1 = real orbital, 0 = padding orbital
 *                 (e.g. the three dummy orbitals of a hydrogen atom); NULL = all
 *                 real.  Padding orbitals must not couple to real ones.
 *   positions     n_block_rows*3 doubles (atom positions) and
 *   box           3 doubles (periodic box lengths); both NULL unless a
 *                 regional solve will be requested.
 *   precision     marnoldi_precision.
 *   cuda_stream   cudaStream_t to issue all work on (NULL = legacy default stream).
 *
 * Checks (MARNOLDI_EINVAL): pattern shape, ascending columns, diagonal blocks,
 * pattern symmetry, |H - H^T| and |S - S^T| <= 1e-12 max|.|, finite values.
 * MARNOLDI_ENOTSPD: S_jj <= 0 for a real orbital, or a Lanczos Ritz value of S
 * <= 0 (which proves S indefinite).  All checks run on the host before any
 * device work.
 */
int marnoldi_setup(marnoldi_ctx **out, int64_t n_block_rows, const int64_t *row_ptr,
                   const int32_t *col_idx, const double *H_vals, const double *S_vals,
                   const uint8_t *orbital_mask, const double *positions, const double *box,
                   int precision, void *cuda_stream);

/*
 * Run the hot path for a set of columns (arXiv:1307.3218, Section 2: the
 * subspaces L_nu^(j) containing e_j, their nu x nu standard eigenproblems, and
 * the Green's function built from the subspace levels and vectors).
 *
 *   columns, ncols  orbital indices to solve (host int64); columns == NULL and
 *                   ncols < 0 select every real orbital.  Duplicates and
 *                   padding orbitals are rejected (MARNOLDI_EINVAL).
 *   nu              subspace dimension, 1 <= nu <= min(M_real, 320); in regional
 *                   mode also nu <= 4 * region_atoms.
 *   region_atoms    0 = global mode (Krylov vectors over all M orbitals, M <= 16384).
 *                   N_reg > 0 = regional mode: column j of atom J is solved on the
 *                   principal sub-pair of (H, S) over the N_reg atoms nearest J
 *                   (squared minimum-image distance, ties to the lower atom index,
 *                   J always included), so M may exceed 16384.  Needs positions
 *                   and box at setup; 1 <= N_reg <= min(n_block_rows, 1024), else
 *                   MARNOLDI_EINVAL.  N_reg = n_block_rows reproduces global mode
 *                   bit for bit.
 *   electron_count  target N_e of the bisection (ignored when mu_fixed != NULL).
 *   kT              > 0.
 *   mu_fixed        NULL = find mu by bisection on N(mu) = sum_j sum_a 2 f w_a over
 *                   the solved columns, bracket [min eps - 40 kT, max eps + 40 kT],
 *                   stop at |N - N_e| <= 1e-12 N_e or after 200 halvings;
 *                   else use *mu_fixed.
 *
 * Per-column Krylov breakdown (||w||_S <= 1e-10 ||H k_n||_S in FP64, 1e-5 in
 * MIXED) is not an error: the column keeps nu_eff < nu levels (see
 * marnoldi_column_stats).  Replaces the previous solve's results.
 */
int marnoldi_solve(marnoldi_ctx *ctx, const int64_t *columns, int64_t ncols, int nu,
                   int region_atoms, double electron_count, double kT, const double *mu_fixed);

/*
 * Density and energy-density values on H's pattern after marnoldi_solve:
 * rho e_j = K V diag(2 f) V^T q and rho^E e_j = K V diag(2 f eps) V^T q with
 * q = K^T e_j (arXiv:1307.3218, Section 2: the Green's function determined by
 * the subspace levels and vectors).  Each output holds nnzb*16 doubles in the
 * BSR layout above; entries of columns that were not solved are set to 0.
 * marnoldi_density writes host arrays, marnoldi_density_device device arrays
 * (written in the context's stream order).
 */
int marnoldi_density(marnoldi_ctx *ctx, double *rho_vals, double *rhoE_vals);
int marnoldi_density_device(marnoldi_ctx *ctx, double *rho_vals_device, double *rhoE_vals_device);

/*
 * Band energy E = sum_j sum_a 2 f eps_a w_a, the Fermi level mu and the
 * electron count N(mu) of the last solve (any pointer may be NULL).
 */
int marnoldi_energy(marnoldi_ctx *ctx, double *band_energy, double *mu, double *electron_count_out);

/*
 * Fermi level of a column set shared by several contexts (arXiv:1307.3218,
 * Section 2: the density is a sum over the columns of all atoms; columns split
 * across contexts or GPUs share one mu).  After marnoldi_solve:
 *   marnoldi_level_range  smallest and largest subspace level of the solved
 *                         columns (host outputs), for the bisection bracket.
 *   marnoldi_fermi_at     N(mu) = sum_j sum_a 2 f((eps_a - mu) / kT) w_a and
 *                         E(mu) = sum_j sum_a 2 f eps_a w_a over this context's
 *                         solved columns, computed on the GPU (outputs may be
 *                         NULL), and makes mu, kT the context's Fermi level for
 *                         marnoldi_density, marnoldi_energy and marnoldi_green.
 * A caller that splits the columns sums N(mu) over the contexts at every
 * bisection step.  Errors: MARNOLDI_EINVAL (null outputs of level_range,
 * kT <= 0 or a non-finite mu), MARNOLDI_ESTATE (no successful solve).
 */
int marnoldi_level_range(marnoldi_ctx *ctx, double *eps_min, double *eps_max);
int marnoldi_fermi_at(marnoldi_ctx *ctx, double mu, double kT, double *N, double *E);

/*
 * Green's-function values G(z) e_j = K V diag(1 / (z - eps)) V^T q on H's
 * pattern (the solution x of (z S - H) x = e_j inside L_nu^(j); Eq. 1 of
 * arXiv:1307.3218) for nz complex shifts z = z_re_im[2i] + i z_re_im[2i+1].
 * G_re_im (host) receives nz * nnzb * 16 complex values, interleaved (re, im),
 * shift-major.  Entries of unsolved columns are 0.
 */
int marnoldi_green(marnoldi_ctx *ctx, const double *z_re_im, int nz, double *G_re_im);

/*
 * Atomic forces F_K = -Tr(rho dH/dR_K) + Tr(rho^E dS/dR_K) from the density and
 * energy-density matrices of the last solve at its Fermi level (arXiv:1307.3218,
 * Section 2: the Green's function gives the total energy and the force; the
 * formula is the standard one for a non-orthogonal basis, with the column
 * results symmetrised, rho_bar = (rho + rho^T) / 2, so that
 * F_K = 2 sum_{J != K} sum_ab (rho_bar_KJ dH_KJ - rho^E_bar_KJ dS_KJ)_ab).
 *   dH_dd, dS_dd  host, [3][nnzb][4][4]: block (I, J) of H and S differentiated
 *                 with respect to d = R_J - R_I along x, y, z (two-centre
 *                 models: dH_IJ/dR_J = +dH_dd, dH_IJ/dR_I = -dH_dd); on-site
 *                 blocks are ignored.
 *   F             host, [n_block_rows][3].
 * Needs a successful solve (MARNOLDI_ESTATE); device scratch of 8 nnzb 16
 * doubles plus F during the call.
 */
int marnoldi_forces(marnoldi_ctx *ctx, const double *dH_dd, const double *dS_dd, double *F);

/*
 * The k-th eigen level and eigenvector from the subspace levels and vectors
 * (arXiv:1307.3218, Section 2, the paragraph on the k-th eigen level, Eq. 3,
 * and the sign rule of the Appendix), after a global-mode marnoldi_solve of
 * every real orbital of one structure (no members).
 *   n(eta) = sum_j sum_a w_a f((eps_a - eta) / sigma) (the integrated density
 *   of states, each level's step smoothed by the Fermi function of width
 *   sigma), eta(n) its inverse by bisection (eta(0) = -inf, eta(M_real) =
 *   +inf), *eps_k = eta(k - 1/2).  phi (host, M doubles; 0 on padding
 *   orbitals and on columns without weight in the window) gets
 *   phi_j = sum_a s_a t_a W_a with t_a = e_j^T K v_a, the window
 *   W_a = f((eps_a - eta(k)) / sigma) - f((eps_a - eta(k-1)) / sigma) (the
 *   smoothed delta of Eq. 3 integrated from eta(k-1) to eta(k)) and the signs
 *   s_a = sign(v_ref^T K v_a) (+1 at 0), v_ref the subspace eigenvector K v_a
 *   (over all M rows) of largest |t_a W_a| over all columns and levels, the
 *   first among equals.  Columns whose largest |t_a W_a| is below 1e-12 of the
 *   reference's are left 0.  eta_bounds (may be NULL): eta(k-1), eta(k).
 * The signs come from a second pass: the reference column's subspace vector by
 * inverse iteration (its nu x nu matrix in shared memory up to nu = 128, else
 * in a device scratch), then a solve of the columns in the window with the
 * projection of their stored vectors on it.  The context's last solve stays.
 * Errors: MARNOLDI_EINVAL (k outside [1, M_real], sigma <= 0, a regional,
 * partial or member solve), MARNOLDI_ESTATE (no solve).
 */
int marnoldi_eigenstate(marnoldi_ctx *ctx, int64_t k, double sigma, double *eps_k, double *phi,
                        double *eta_bounds);

/*
 * Per-column results of the last solve, in the order of the solved columns
 * (host arrays; any may be NULL): nu_eff[ncols], eps[ncols*nu] (ascending
 * subspace levels, zero past nu_eff), w[ncols*nu] (weights
 * w_a = sqrt(S_jj) v_a[0] (V^T q)_a, zero past nu_eff).
 */
int marnoldi_column_stats(marnoldi_ctx *ctx, int32_t *nu_eff, double *eps, double *w);

/* Number of solved columns and nu of the last solve (either pointer may be NULL). */
int marnoldi_solved_shape(marnoldi_ctx *ctx, int64_t *ncols, int *nu);

/*
 * Tuning and instrumentation.
 *   marnoldi_set_batch: columns per device batch (0 = choose from free memory).
 *     In regional mode a batch smaller than the column list is rounded down to
 *     a multiple of 4, so that the orbitals of one atom, listed together, stay
 *     in one batch (they share the regional product's block reads).
 *   marnoldi_set_profiling: 1 = time every kernel launch with CUDA events on the
 *     context's stream (adds event records; off by default).
 *   marnoldi_kernel_stats: for kind = 0 .. marnoldi_kernel_kinds()-1, the kernel
 *     name, the number of launches and the summed event time (ms, profiling
 *     only) since the last reset; reset != 0 clears them after reading.
 *   marnoldi_set_krylov_graph: 1 = run the Krylov build of every batch (support
 *     search, initial vectors, nu steps of product and Gram-Schmidt: 2 nu + 2
 *     or 2 nu + 3 kernels) as one CUDA graph, captured from the context's
 *     stream and launched once; the executable graph is kept in the context and
 *     updated in place for the next batch or solve with the same nu and mode.
 *     Not while profiling is on (kernels are then launched and timed one by
 *     one).  The same kernels with the same arguments run in the same order,
 *     so results equal the direct launches bit for bit.  The default for a new
 *     context is 1 when the environment variable MARNOLDI_KRYLOV_GRAPH is "1",
 *     else 0.  MARNOLDI_EINVAL for other values.
 *   marnoldi_krylov_graph_launches: graphs launched by this context so far.
 */
int marnoldi_set_batch(marnoldi_ctx *ctx, int64_t batch_columns);
int marnoldi_set_profiling(marnoldi_ctx *ctx, int enable);
int marnoldi_set_krylov_graph(marnoldi_ctx *ctx, int enable);
int marnoldi_krylov_graph_launches(const marnoldi_ctx *ctx, int64_t *graph_launches);
int marnoldi_kernel_kinds(void);
int marnoldi_kernel_stats(marnoldi_ctx *ctx, int kind, const char **name, int64_t *launches,
                          double *ms, int reset);

/*
 * Members: one context holding several independent structures as a
 * block-diagonal union, solved in the same kernel launches (one launch per
 * step covers the columns of every member), each member with its own
 * electron count and Fermi level.
 *   marnoldi_set_members(ctx, n, atom_offsets[n + 1], electron_counts[n])
 *     Member q is atoms [atom_offsets[q], atom_offsets[q + 1]); offsets run
 *     from 0 to n_block_rows, every member starts at a multiple of 8 atoms (pad
 *     with atoms whose four orbitals are padding orbitals), and no block may
 *     couple two members (MARNOLDI_EINVAL otherwise).  n = 0 removes the
 *     members.  Clears the last solve.
 *   A marnoldi_solve of a context with members takes every real orbital
 *   (columns = NULL), global mode, nu <= 253 and mu by bisection (mu_fixed =
 *   NULL; electron_count is ignored): each member's mu solves N(mu) = its
 *   electron count over its own columns with the usual bracket and rule.  The
 *   Krylov vectors are as long as the largest member needs, so a member solved
 *   in a union whose largest member has the same padded length gets the same
 *   results as alone, bit for bit.  marnoldi_density, _density_device, _forces
 *   and _green use each member's own mu; marnoldi_energy returns the sums of
 *   E_band and N over the members (mu of member 0); marnoldi_level_range and
 *   marnoldi_fermi_at return MARNOLDI_EINVAL.
 *   marnoldi_member_energy(ctx, q, ...): E_band, mu and N(mu) of member q.
 *   marnoldi_set_member_temperatures(ctx, n, kT[n]): member q's Fermi level,
 *     density and energy use kT[q] (> 0, finite) instead of the solve's kT;
 *     n must equal the member count (MARNOLDI_EINVAL otherwise).  kT enters
 *     only the Fermi step, so members of different temperatures share every
 *     Krylov launch.  marnoldi_set_members clears the temperatures; this call
 *     clears the last solve.
 */
int marnoldi_set_members(marnoldi_ctx *ctx, int n_members, const int64_t *atom_offsets,
                         const double *electron_counts);
int marnoldi_member_energy(marnoldi_ctx *ctx, int member, double *band_energy, double *mu,
                           double *electron_count_out);
int marnoldi_set_member_temperatures(marnoldi_ctx *ctx, int n_members, const double *kT);

/*
 * Launch-shape autotuner of the Gram-Schmidt kernel (process-wide).
 *   marnoldi_set_autotune: mode 0 (default, also when MARNOLDI_AUTOTUNE is
 *     unset or not "1") uses a fixed rule: 256 threads per CTA up to m = 4096,
 *     512 for FP32 vectors up to 8192, the streamed kernel for longer FP32
 *     vectors (reported as 64 values per thread and 288 threads: 256
 *     threads and a producer warp that copies the vectors into shared memory
 *     with the bulk-copy engine), else 1024, values per thread covering m.
 *     Mode 1: the first solve of each (precision, nu, global/regional, padded
 *     vector length) times every shape with the same padded length (threads
 *     256, 512 or 1024; for FP32 vectors of 16,384 entries also the two
 *     streamed shapes, 64 x 288 and 32 x 544: 512 consumer threads and the
 *     producer, one CTA per SM) on its first 1,216 columns, keeps the fastest for the
 *     rest of the process and, when MARNOLDI_TUNE_CACHE names a file, appends
 *     it there and reads earlier choices from it.  Shapes change the order of
 *     the kernel's partial sums, so results may differ by rounding between
 *     shapes (within the solve's accuracy); a shape once chosen stays fixed.
 *     MARNOLDI_EINVAL for other modes.
 *   marnoldi_gs_shape: values per thread and threads per CTA of the last solve
 *     (0, 0 before the first).
 */
int marnoldi_set_autotune(int mode);
int marnoldi_gs_shape(const marnoldi_ctx *ctx, int *values_per_thread, int *threads);

/*
 * Index checks (debugging).  A library built with -DMARNOLDI_CHECK (the build
 * script's "check" variant) tests, in its kernels, the indices that come from
 * data (block lists, tile orders, support counts, output offsets) before
 * using them; a failed test skips the access and records the first failure of
 * its source file, and no kernel ever traps.  marnoldi_check_status reports
 * *compiled = 1 in such a build (0 otherwise, with *site = 0), the first
 * recorded failure as *site (a CheckSite number, 0 = none) and *index (the
 * offending index), and clears the records.  It synchronises with the device.
 * Errors (MARNOLDI_EINVAL, MARNOLDI_ECUDA) through marnoldi_last_error(NULL).
 */
int marnoldi_check_status(int *compiled, int *site, int64_t *index);

/*
 * Electron count and band energy at a given mu over subspace levels already in
 * device memory, without allocating any device memory.  The paper has no
 * counterpart: this is a variant of the bisection's reduction for callers that
 * cannot call cudaMalloc (code running under another framework's memory
 * manager, or on a request path that must not allocate).
 *
 *   eps_device, w_device  ncols*nu doubles each (levels and weights, the layout
 *                         of marnoldi_column_stats).
 *   nu_eff_device         ncols int32 valid-level counts, or NULL (all nu valid).
 *   out_device            2 doubles: N(mu) = sum 2 f w, E(mu) = sum 2 f eps w.
 *   cuda_stream           stream to run on (NULL = legacy default stream).
 *
 * Scratch: a fixed 64 KiB device array inside the library (every GPU that
 * loads the library holds it until exit), so ncols*nu is limited to
 * MARNOLDI_COUNT_NOALLOC_MAX_LEVELS = 16,777,216 levels; larger inputs return
 * MARNOLDI_EINVAL.  Every call looks up that array's device address on the
 * current device (no allocation); the first call on a device also loads the
 * library's device code there, so make it before any stream capture.
 * Every call shares the one array: calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller.
 * Errors are reported through marnoldi_last_error(NULL).
 */
#define MARNOLDI_COUNT_NOALLOC_MAX_LEVELS 16777216
int marnoldi_count_noalloc(const double *eps_device, const double *w_device,
                           const int32_t *nu_eff_device, int64_t ncols, int nu, double mu,
                           double kT, double *out_device, void *cuda_stream);

/*
 * Device memory.
 *   marnoldi_device_bytes: bytes the context holds now and the most it has held
 *     since setup (requested sizes; the allocator may round them up).
 *   marnoldi_footprint: the peak of marnoldi_setup, one marnoldi_solve of every
 *     real orbital (columns == NULL) and one marnoldi_density, computed on the
 *     host from the block pattern alone: structure copies, column state, batch
 *     workspace of batch_columns columns (>= 1; clamped to the column count and
 *     the launch limits, and in regional mode rounded down to a multiple of 4
 *     when below the column count; the value used goes to *batch_used, which
 *     may be NULL)
 *     and the density staging.  box is needed in regional mode (cell list).  It
 *     equals the peak of marnoldi_device_bytes of such a run.  Errors
 *     (MARNOLDI_EINVAL, through marnoldi_last_error(NULL)): arguments that
 *     marnoldi_setup or marnoldi_solve would reject on size grounds.
 */
int marnoldi_device_bytes(const marnoldi_ctx *ctx, size_t *current, size_t *peak);
int marnoldi_footprint(int64_t n_block_rows, const int64_t *row_ptr, const uint8_t *orbital_mask,
                       const double *box, int precision, int nu, int region_atoms,
                       int64_t batch_columns, size_t *bytes, int64_t *batch_used);

/*
 * Request server: whole calculations (setup, solve of every real orbital with
 * the bisection on N_e, density and energy-density matrices, band energy) on
 * structures of any size and nu, submitted at any time from any thread and run
 * concurrently on the current CUDA device.
 *
 *   marnoldi_server_create(out, workers, hbm_budget_bytes)
 *     `workers` threads (1..64), each with its own non-blocking stream, take
 *     requests in submission order.  A request starts when a worker is free and
 *     its footprint (marnoldi_footprint) fits under hbm_budget_bytes beside the
 *     footprints of the running requests.  Device memory comes from a pool of
 *     the server that keeps up to the budget mapped between requests.
 *   marnoldi_server_submit(...)
 *     Arguments as marnoldi_setup and marnoldi_solve (mu always by bisection).
 *     batch_columns 0 = the largest batch whose footprint stays within
 *     budget / workers (at least one column).  rho_vals, rhoE_vals: host arrays
 *     of nnzb*16 doubles that receive the density and energy-density matrices
 *     (both NULL = energy only).  Every array passed must stay valid and
 *     unchanged until marnoldi_server_wait has returned this request's result.
 *     Returns MARNOLDI_ENOMEM when the footprint exceeds the whole budget,
 *     MARNOLDI_EINVAL for arguments the footprint check rejects and for
 *     kT or electron_count not positive and finite; other input
 *     errors come back as the request's status.  *request_id > 0 on success.
 *   marnoldi_server_wait(srv, id, timeout_s, status, result, message, cap)
 *     Waits up to timeout_s seconds (< 0 = no limit).  MARNOLDI_EPENDING if the
 *     request is still queued or running (it stays waitable); MARNOLDI_EINVAL
 *     for an unknown id; else MARNOLDI_OK, and the request's record is
 *     released after writing (any output may be NULL):
 *       *status    the request's marnoldi_status,
 *       result[8]  band energy, mu, N(mu), then the submit, start and end
 *                  times (seconds on the server's steady clock), the footprint
 *                  in bytes and the batch size,
 *       message    the request's error message (empty on success), truncated
 *                  to cap - 1 characters.
 *   marnoldi_server_stats(srv, stats[9])
 *     queued, running, completed, footprint bytes in use, most footprint bytes
 *     in use at once, most launch groups running at once, the pool's most
 *     reserved bytes, groups of two or more requests formed, the largest group.
 *   marnoldi_server_set_group_limit(srv, n)
 *     Continuous batching: when a worker starts a request, up to n - 1 queued
 *     requests of the same precision, nu and kT, global mode, nu <= 253, whose
 *     Krylov vectors have the same padded length (and that all want or all skip
 *     the density) join it as members of one context (marnoldi_set_members;
 *     union <= 4,096 atoms), while the union's footprint fits beside the running
 *     requests.  Each member's results equal its results alone, bit for bit.
 *     Default 16; 1 runs every request on its own.  MARNOLDI_EINVAL outside
 *     [1, 64].  For members of a group, result[6] and result[7] of
 *     marnoldi_server_wait are the group's footprint and batch.
 *   marnoldi_server_destroy(srv)
 *     Waits for every submitted request to finish, then frees the workers,
 *     streams and pool.  Records never waited for are dropped.
 * Errors of create, submit, wait and stats: marnoldi_server_last_error()
 * (per calling thread).
 */
typedef struct marnoldi_server marnoldi_server;
int marnoldi_server_create(marnoldi_server **out, int workers, size_t hbm_budget_bytes);
int marnoldi_server_submit(marnoldi_server *srv, int64_t n_block_rows, const int64_t *row_ptr,
                           const int32_t *col_idx, const double *H_vals, const double *S_vals,
                           const uint8_t *orbital_mask, const double *positions, const double *box,
                           int precision, int nu, int region_atoms, double electron_count, double kT,
                           int64_t batch_columns, double *rho_vals, double *rhoE_vals,
                           int64_t *request_id);
int marnoldi_server_wait(marnoldi_server *srv, int64_t request_id, double timeout_s, int *status,
                         double *result, char *message, size_t message_cap);
int marnoldi_server_stats(marnoldi_server *srv, int64_t *stats);
int marnoldi_server_set_group_limit(marnoldi_server *srv, int max_members);
const char *marnoldi_server_last_error(void);
void marnoldi_server_destroy(marnoldi_server *srv);

/* Message of the last failure on ctx (or of the last failed setup when ctx is NULL). */
const char *marnoldi_last_error(const marnoldi_ctx *ctx);

/* Release the context and its device memory (NULL is ignored). */
void marnoldi_destroy(marnoldi_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* MARNOLDI_H */
