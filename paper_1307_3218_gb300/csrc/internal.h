// Internal declarations shared by the libmarnoldi translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "marnoldi.h"

namespace marnoldi {

// Kernel kinds, for launch counting and optional event timing.
enum KernelKind {
    KK_INIT = 0,
    KK_SPMM_H,
    KK_GS,
    KK_SPMM_S,
    KK_EIG,
    KK_MINMAX,
    KK_COUNT,
    KK_DENSITY,
    KK_GREEN,
    KK_REGION,
    KK_SUPPORT,
    KK_SPMM_HS,
    KK_BISECT,
    KK_FORCE,
    KK_EIGSTATE,
    KK_NKINDS
};

const char *kernel_name(int kind);

// Record the message that marnoldi_last_error(NULL) returns; returns `code`.
int set_global_error(int code, const char *msg);

// marnoldi_setup with the context's own device allocator in place of the
// process-wide hook (the request server draws each request's memory from its
// own pool).  alloc == NULL selects cudaMallocAsync / cudaFreeAsync.
int setup_with_allocator(marnoldi_ctx **out, int64_t n_block_rows, const int64_t *row_ptr,
                         const int32_t *col_idx, const double *H_vals, const double *S_vals,
                         const uint8_t *orbital_mask, const double *positions, const double *box,
                         int precision, void *cuda_stream, marnoldi_alloc_fn alloc,
                         marnoldi_free_fn free_fn, void *user);

// What a solve's memory depends on, from a block pattern: block rows, blocks,
// real orbitals (columns), their pattern rows, the longest block row, and the
// Krylov-vector length (4 n_block_rows; for a union of structures, 4 x the
// largest member's span).
struct PatternStats {
    int64_t nbr = 0, nnzb = 0, nc = 0, prow = 0, m_vec = 0;
    int maxrow = 1;
};
int pattern_stats(int64_t n_block_rows, const int64_t *row_ptr, const uint8_t *orbital_mask, PatternStats &st);
// marnoldi_footprint from the statistics (every real orbital solved).
int footprint_of(const PatternStats &st, int precision, int nu, int region_atoms, const double *box,
                 int64_t batch_columns, size_t *bytes, int64_t *batch_used);

// Let `kernel` launch with up to `bytes` of dynamic shared memory.  The limit
// only grows, and callers on several threads may race: one lock orders them.
cudaError_t allow_dynamic_smem(const void *kernel, size_t bytes);

// Largest subspace dimension.  Up to about 110 the subspace matrix of the
// eigensolve sits in shared memory, above that in a global scratch.
constexpr int kMaxNu = 320;
// Largest Krylov-vector length of global mode (one CTA holds a column's vector).
constexpr int64_t kMaxGlobalM = 16384;

// Threads per CTA and values per thread of the column-per-CTA kernels on
// vectors of length m: m_pad = vpt * threads >= m, a multiple of 32.
struct ColumnShape {
    int vpt;
    int threads;
    int64_t m_pad;
};
ColumnShape column_shape(int64_t m, int prec);
// Every shape the Gram-Schmidt kernels are built for with the same m_pad and
// precision (threads 256, 512 or 1024; at most kMaxShapes); returns how many
// were written.
constexpr int kMaxShapes = 4;
int column_shape_candidates(int64_t m_pad, int prec, ColumnShape *out);
// The shapes of the streamed Gram-Schmidt kernel (gs_stream.cu), FP32
// vectors of m_pad = 16,384 and a producer warp: 512 consumer threads of 32
// values, {vpt 32, threads 544}, or 256 of 64 values, {vpt 64, threads 288}.
bool gs_stream_shape(const ColumnShape &s, int prec);

// ---------------------------------------------------------------- Krylov build
// All pointers are device pointers.  Batch layout (c = batch column):
//   K[c][i][r], SK[c][i][r] at ((c * nu) + i) * m_pad + r  (i < nu): the
//     basis vectors *unnormalised*, w_i and S w_i; the S-orthonormal basis is
//     k_i = scale[c][i] * w_i (scale = 1 / ||w_i||_S, set by the MGS of step i)
//   U[c][r] at c * m_pad + r: H w_n of the current step
//   Hsub[c][i][l] at (c * nu + i) * nu + l (double)
// status[c]: 0 active, 1 stopped (breakdown), 2 non-positive S norm, 3 a bounded
// wait of the streamed Gram-Schmidt kernel gave up.
struct KrylovBatch {
    int prec;             // 0 FP64, 1 mixed (vectors float)
    int nb;               // columns in this batch
    int nu;
    int64_t m;            // vector length
    ColumnShape shape;
    void *K, *SK, *U;
    void *Ulo;            // mixed precision: lo word of H w_n (u = U + Ulo to ~2^-48)
    double *Hsub;         // [c][nu][nu]: k_i . H k_l of the stored basis (unit S-norm)
    double *Lsub;         // [c][nu][nu]: L^-1, L the lower Cholesky factor of its S-Gram matrix
    double *scale;        // [c][nu]
    double *cn2;          // per column: |S-projection of s_n H w_n on the basis|_S^2 of the last step
    int *status;
    int *nu_eff;
    const int64_t *cols;  // global orbital column of each batch column
    // Structural support of the basis, over tiles of 8 atoms (32 vector
    // entries; t < ntile = m_pad / 32):
    //   thop[t * nb + c]          fewest pattern hops from the column's atom to
    //                             an atom of tile t (255: more than nu + 1)
    //   tinv[t * nb + c]          position of tile t in column c's tile order,
    //                             (thop, t) ascending
    //   tcnt[c * (nu + 2) + L]    number of tiles with thop <= L (L <= nu + 1)
    // Column c's vectors (K, SK, U, Ulo) are stored in its tile order: entry r
    // at position vpos(r) = 32 tinv[r / 32] + r % 32.  w_i vanishes outside
    // the first tcnt[i] tiles, S w_i and H w_i outside the first tcnt[i + 1].
    // ntile (tiles of the structure) is at least m_pad / 32; it is larger for
    // a union of structures, whose columns only ever use their own tiles.
    int ntile = 0;
    uint8_t *thop = nullptr;
    uint16_t *tinv = nullptr;
    int *tcnt = nullptr;
};

// ---------------------------------------------------------------- index checks
// Built with -DMARNOLDI_CHECK, kernels test the indices they take from data
// (block lists, tile orders, support counts, output offsets) before using
// them.  A failed test records the first failure of its translation unit
// (the check site and the index) in a device word and the access is skipped:
// nothing traps.  marnoldi_check_status reads and clears the words.  Without
// the flag every test is the constant true and compiles away.
enum CheckSite : int {
    kChkSpmmGather = 1,   // krylov.cu: position of a gathered 4-vector in a column's vector
    kChkInitPos,          // krylov.cu: position of an entry of S e_j
    kChkRegionCol,        // region.cu: local column of a local block
    kChkRegionGather,     // region.cu: position of a gathered 4-vector
    kChkDensityOut,       // outputs.cu: density entry of a pattern row
    kChkSupportCount,     // krylov.cu, gs_stream.cu: tiles of a support (at most m_pad / 32)
};
#ifdef MARNOLDI_CHECK
constexpr bool kCheckBuild = true;
namespace {
__device__ unsigned long long g_check_word;   // one per translation unit
__device__ __forceinline__ bool in_range(int64_t i, int64_t n, int site)
{
    if (i >= 0 && i < n) return true;
    atomicCAS(&g_check_word, 0ull,
              (1ull << 63) | ((unsigned long long)(site & 0x7fff) << 40) | ((unsigned long long)i & 0xffffffffffull));
    return false;
}
}  // namespace
// Defines check_take_<name>: read this translation unit's word and clear it.
#define MARNOLDI_CHECK_TAKE(name)                                                       \
    cudaError_t check_take_##name(unsigned long long *w)                                \
    {                                                                                   \
        cudaError_t e = cudaMemcpyFromSymbol(w, g_check_word, sizeof(*w));             \
        if (e == cudaSuccess && *w) {                                                   \
            const unsigned long long z = 0;                                             \
            e = cudaMemcpyToSymbol(g_check_word, &z, sizeof(z));                        \
        }                                                                               \
        return e;                                                                       \
    }
#else
constexpr bool kCheckBuild = false;
__device__ __forceinline__ constexpr bool in_range(int64_t, int64_t, int) { return true; }
#define MARNOLDI_CHECK_TAKE(name)                            \
    cudaError_t check_take_##name(unsigned long long *w)     \
    {                                                        \
        *w = 0;                                              \
        return cudaSuccess;                                  \
    }
#endif
cudaError_t check_take_krylov(unsigned long long *w);
cudaError_t check_take_region(unsigned long long *w);
cudaError_t check_take_outputs(unsigned long long *w);
cudaError_t check_take_gs_stream(unsigned long long *w);

// Four consecutive values (16-byte aligned for float, 32 for double) in one or
// two vector loads (read-only path) or stores.
__device__ __forceinline__ void load4(const double *p, double (&v)[4])
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load4(const float *p, float (&v)[4])
{
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void store4(double *p, const double (&v)[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void store4(float *p, const float (&v)[4])
{
    reinterpret_cast<float4 *>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
}

// Storage position of vector entry r of batch column c (see KrylovBatch).
__device__ __forceinline__ int64_t vpos(const uint16_t *__restrict__ tinv, int nb, int c, int64_t r)
{
    return 32 * (int64_t)tinv[(r >> 5) * nb + c] + (r & 31);
}
constexpr int kMaxTiles = (int)(kMaxGlobalM / 32);

struct DeviceMatrix {
    int64_t nbr, nnzb;
    const int64_t *rp;
    const int32_t *ci;
    const double *Hd, *Sd;   // FP64 values
    // Mixed precision: per block 16 "hi" then 16 "lo" FP32 values with
    // hi + lo = the FP64 value to about 2^-48 (else null).
    const float *Hf, *Sf;
    const double *sdiag;     // S_jj, length 4 nbr
    const int64_t *tmap;     // block (J, I) -> index of block (I, J)
};

// ---------------------------------------------------------------- regional mode
// Per batch column c: reg[c][p] (region atoms, ascending), lcnt[c][p] local
// blocks of local row p, lci/lgk[c][slot][p] their local column and global
// block index; rstat[c] 0 ok, 1 fewer than n_reg atoms within r_s, 2 more
// candidates than kRegionCap.
constexpr int kRegionCap = 8192;      // candidates per region search (power of two)
constexpr int kMaxRegion = 1024;      // n_reg limit (local vectors <= 4096)
struct RegionMaps {
    int n_reg = 0, maxrow = 0;
    const double *pos = nullptr, *box = nullptr;
    const int *cell_start = nullptr, *cell_atoms = nullptr;
    int ncell[3] = {1, 1, 1};
    double cell_edge[3] = {1.0, 1.0, 1.0};
    int *reg = nullptr, *lcnt = nullptr, *lci = nullptr, *lgk = nullptr, *rstat = nullptr;
    // the batch's groups of the regional product: group g is batch columns
    // gstart[g] .. gstart[g + 1] - 1, one atom's, at most regional_group(prec)
    const int *gstart = nullptr;
    int ngroups = 0;
};

// Columns per group of the regional product (the columns of one atom that
// share a pass over the local blocks): 4 in mixed precision, 2 in FP64.
int regional_group(int prec);

cudaError_t launch_region(const RegionMaps &rm, const KrylovBatch &b, double rs, int cap,
                          cudaStream_t s);
cudaError_t launch_local_bsr(const DeviceMatrix &A, const RegionMaps &rm, const KrylovBatch &b,
                             cudaStream_t s);
cudaError_t launch_init_regional(const DeviceMatrix &A, const RegionMaps &rm, const KrylovBatch &b,
                                 cudaStream_t s);
// H x (to b.U, b.Ulo) and, when SY is given, S x (to SY) in one pass over the
// local block lists, with the sums of the separate products.
cudaError_t launch_spmm_regional_hs(const DeviceMatrix &A, const RegionMaps &rm, const KrylovBatch &b,
                                    const void *X, int64_t ldx, void *SY, int64_t ldsy, int lim,
                                    cudaStream_t s);

// Position of atom a in the ascending list R[0..n), or -1.
__device__ __forceinline__ int find_sorted(const int *__restrict__ R, int n, int a)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (R[mid] < a) lo = mid + 1; else hi = mid;
    }
    return (lo < n && R[lo] == a) ? lo : -1;
}

cudaError_t launch_init(const DeviceMatrix &A, const KrylovBatch &b, cudaStream_t s);
// Fills thop / tinv / tcnt of the batch (rm = null in global mode).
// Zeros at the positions of the rows past `rows` (atoms, or region atoms) in
// their last tile of 8, in U, Ulo and the S w slots of every batch column; a
// no-op when rows is a multiple of 8.
cudaError_t launch_zero_partial_tile(const KrylovBatch &b, int rows, cudaStream_t s);
cudaError_t launch_support(const DeviceMatrix &A, const RegionMaps *rm, const KrylovBatch &b,
                           cudaStream_t s);
// U (and Ulo) = H X and, when SY is not null, SY = S X for the batch (X and
// SY with column strides ldx, ldsy; U with m_pad); rows of tiles with
// thop > lim are written as zeros without being computed (X must vanish
// outside thop <= lim - 1).
cudaError_t launch_spmm_hs(const DeviceMatrix &A, const KrylovBatch &b, const void *X, int64_t ldx,
                           void *SY, int64_t ldsy, int lim, cudaStream_t s);
cudaError_t launch_gs(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s);
cudaError_t launch_gs_stream(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s);

// ---------------------------------------------------------------- subspace eigensolve
// Per solved column c (global index col0 + batch column):
//   eps/w/t at c * nu (zero past nu_eff); P rows at p_off[c] (n_pat x nu, row-major).
struct ColumnState {
    int64_t ncols;
    int nu;
    const int64_t *cols;
    int *nu_eff;
    double *eps, *w, *t, *P;
    const int64_t *p_off;
    int *eig_status;     // bits: 1 QL did not converge, 2 non-positive S norm, 4 a wait gave up
};

// Scratch of the three-kernel eigensolve, per chunk of subspaces:
//   D, E [chunk][nu] (tridiagonal, then levels), RQ [chunk][nr_max][nu] (rows
//   e_1, q, K_pat times Q, then times Z), rot [chunk][rcap] Givens (c, s),
//   sweep [chunk][scap] (m, lo), nsweep [chunk] (-1: QL failed).
struct EigScratch {
    int chunk = 0, nr_max = 0;
    int64_t rcap = 0, scap = 0;
    double *D = nullptr, *E = nullptr, *RQ = nullptr;
    double2 *rot = nullptr;
    int2 *sweep = nullptr;
    int *nsweep = nullptr;
    double *Ag = nullptr;   // chunk x nu x (nu | 1) doubles when H_sub does not fit in shared memory
    // optional extra row of R: proj[c * nu + i] = v^T w_i (batch column c, stored
    // vector i) for a given vector v; the eigensolve then writes v^T K v_a of
    // every level a (ascending) to proj_out[g * nu + a] (g = solved column)
    const double *proj = nullptr;
    double *proj_out = nullptr;
};
// Dynamic shared memory of the tridiagonalisation and the largest one of the
// eigensolve kernels, with H_sub in shared (a_global = false) or global memory.
size_t eig_tridiag_smem(int nu, int nr_max, bool a_global);
size_t eig_smem_bytes(int nu, int nr_max, bool a_global);

cudaError_t launch_eig(const DeviceMatrix &A, const KrylovBatch &b, const ColumnState &st,
                       int64_t col0, const RegionMaps *rm /* null in global mode */,
                       const EigScratch &es, cudaStream_t s);

// ---------------------------------------------------------------- Fermi level, outputs
// Deterministic two-level reductions; `partial` holds 2 * kReduceBlocks doubles,
// `ticket` one zero-initialised unsigned int, `out` two doubles.
constexpr int kReduceBlocks = 304;
cudaError_t launch_minmax(const ColumnState &st, double *partial, unsigned *ticket, double *out,
                          cudaStream_t s);
// Fermi-level bisection on the device: bracket [min eps - 40 kT, max eps + 40 kT],
// stop at |N - N_e| <= 1e-12 N_e or after 200 halvings.
constexpr double kBisectBracketKT = 40.0;
constexpr double kBisectRtol = 1e-12;
constexpr int kBisectMaxit = 200;
struct BisectState {
    double lo, hi, mu, N, E, Nlo, Nhi;
    int it, phase, status, steps;   // status 1: N_e outside [N(lo), N(hi)]
};
// Level range into range[0..1], then a CUDA graph with a while node that
// alternates bisect_step_kernel and count_kernel (mu read from bs->mu) until
// the step ends the loop; bs holds the result once the stream reaches it.
cudaError_t launch_bisection(const ColumnState &st, double kT, double electron_count, double *partial,
                             unsigned *ticket, double *range, double *out, BisectState *bs,
                             cudaStream_t s);
// The k-th eigen level and vector (eigstate.cu).
//   launch_window   colmax[c] = max_a |t_a W_a|, colarg[c] its level, argmax[0] the column
//                   of the largest (W_a = f((eps_a - hi) / sigma) - f((eps_a - lo) / sigma))
//   launch_project  proj[c * nu + i] = v^T w_i for the batch's stored vectors (v over M rows)
//   launch_eigvec   out[r] (M rows, untouched outside the column's tiles) = row r of K v_a for
//                   the level eps of batch column c (nu <= eigvec_max_nu(); Ag: a scratch of
//                   eigvec_scratch_bytes(nu) bytes, needed above 128)
//   launch_combine  phi[cols[c]] = sum_a sign(proj[c nu + a]) t_a W_a over the solved columns
cudaError_t launch_window(const ColumnState &st, double lo, double hi, double sigma, double *colmax, int *colarg,
                          int64_t *argmax, cudaStream_t s);
cudaError_t launch_project(const KrylovBatch &b, const double *v, int64_t M, double *proj, cudaStream_t s);
int eigvec_max_nu();
size_t eigvec_scratch_bytes(int nu);
cudaError_t launch_eigvec(const KrylovBatch &b, int c, double eps, int64_t M, double *out, double *Ag,
                          cudaStream_t s);
cudaError_t launch_combine(const ColumnState &st, const double *proj, double lo, double hi, double sigma,
                           double *phi, cudaStream_t s);

// F[n_atoms][3] = 2 sum_J sum_ab (rho_bar dH - rho_bar^E dS) over the blocks
// (K, J != K); rho, rhoE, dH, dS device arrays in the BSR layout (dH, dS
// [3][nnzb][16]).
cudaError_t launch_forces(const DeviceMatrix &A, const double *rho, const double *rhoE, const double *dH,
                          const double *dS, double *F, cudaStream_t s);
cudaError_t launch_count(const ColumnState &st, double mu, double kT, double *partial,
                         unsigned *ticket, double *out, cudaStream_t s);
cudaError_t launch_density(const DeviceMatrix &A, const ColumnState &st, double mu, double kT,
                           double *rho, double *rhoE, cudaStream_t s);
cudaError_t launch_green(const DeviceMatrix &A, const ColumnState &st, double zr, double zi,
                         double *G, cudaStream_t s);

}  // namespace marnoldi
