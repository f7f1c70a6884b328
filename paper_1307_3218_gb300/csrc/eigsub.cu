// Subspace eigensolve of the multiple Arnoldi method on sm_103a.
//
// Each subspace L_nu^(j) gives a nu x nu standard eigenproblem
// H_sub v_a = eps_a v_a whose levels and vectors determine the Green's
// function (arXiv:1307.3218, Section 2).  The outputs need only
//   eps (ascending), V[0][:] and t = V^T q (q = K^T e_j), and P_j = K_pat V,
// i.e. the rows R = [e_1^T; q^T; K_pat] (n_pat + 2 rows) times V.
//
// H_sub is reduced to tridiagonal form T = Q^T H_sub Q by Householder
// reflections and T = Z Lambda Z^T by the implicit-shift QL algorithm
// (Bowdler, Martin, Reinsch & Wilkinson 1968), so R V = (R Q) Z.  Three
// kernels per chunk of subspaces:
//   eig_tridiag_kernel  one CTA per subspace: the reflections, applied to H_sub
//                       and to R (never forming Q); writes d, e and R Q
//   eig_ql_kernel       one LANE per subspace (32 subspaces per warp): the
//                       QL recurrence, which is a serial chain of FP64
//                       divisions and square roots per subspace.  Running 32
//                       chains side by side fills GB300's narrow FP64 pipe
//                       instead of issuing one useful lane per instruction.
//                       Every Givens rotation (c, s) and every sweep's
//                       index range is logged.
//   eig_apply_kernel    one CTA per subspace: each thread replays the log on
//                       its rows of R Q, then the levels are ranked and
//                       eps, w_a = sqrt(S_jj) (R V)[0][a] (R V)[1][a], t and
//                       P_j are written in ascending order of eps.
#include "internal.h"

#include <math_constants.h>

#include <algorithm>
#include <cfloat>

namespace marnoldi {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTriThreads = 256;
constexpr int kApplyThreads = 128;
constexpr int kQlMaxIter = 30;      // QL iterations per eigenvalue

__device__ __forceinline__ double warp_sum(double s)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    return s;
}


// ------------------------------------------------------------------ tridiagonalisation
// A = Q T Q^T with Q = P_0 P_1 ... P_{n-3}; R <- R P_0 P_1 ... (R Q).
// A is symmetric: after the L^-1 transform only its lower triangle is formed
// and updated (the product A v reads it by rows left of the diagonal and by
// columns below), which halves the FP64 work of the rank-2 updates and saves
// two thirds of the second transform's.
// Shared memory: A [n][lda], R [nr_max][lda] (lda = nu | 1, odd, so that the
// per-thread row walks of R spread over the banks), v, e, scalars.  When A
// does not fit (nu above about 110), it lives in a global scratch of
// nu x lda doubles per subspace (Ag), which the CTA's sweeps keep in L2
// (720 KB at nu = 300), and shared memory holds R and the vectors only.
template <typename VT>
__global__ void __launch_bounds__(kTriThreads) eig_tridiag_kernel(
    const double *__restrict__ Hsub, const int *__restrict__ bnu_eff,
    const double *__restrict__ bscale, const VT *__restrict__ K, int64_t m_pad,
    const uint16_t *__restrict__ tinv, int nb, int nu,
    const int64_t *__restrict__ bcols, const int64_t *__restrict__ rp,
    const int32_t *__restrict__ ci, const int *__restrict__ reg, int n_reg, int cofs,
    double *__restrict__ D, double *__restrict__ E, double *__restrict__ RQ, int nr_max,
    double *__restrict__ Ag, const double *__restrict__ Lsub, const double *__restrict__ proj)
{
    const int sc = blockIdx.x;
    const int c = cofs + sc;
    const int n = bnu_eff[c];
    const int tid = threadIdx.x, T = blockDim.x;
    const int lda = nu | 1;
    extern __shared__ __align__(16) double sm[];
    double *A = Ag ? Ag + (size_t)sc * nu * lda : sm;
    double *R = Ag ? sm : A + (size_t)nu * lda;
    double *v = R + (size_t)nr_max * lda;
    double *ev = v + nu;
    __shared__ double sc4[4];
    __shared__ int skip;

    // rows of R: e_1, q = K^T e_j, and K_pat (zero for atoms outside a region)
    const int64_t j = bcols[c];
    const int64_t J = j >> 2;
    const int *Rg = reg ? reg + (int64_t)c * n_reg : nullptr;
    const int pJ = Rg ? find_sorted(Rg, n_reg, (int)J) : 0;
    const int64_t jl = Rg ? 4 * (int64_t)(pJ < 0 ? 0 : pJ) + (j & 3) : j;
    const int64_t kb = rp[J];
    const int npat = 4 * (int)(rp[J + 1] - kb);
    const int nr = npat + 2 + (proj ? 1 : 0);   // the projection row last
    const VT *Kc = K + (int64_t)c * nu * m_pad;
    for (int idx = tid; idx < n * n; idx += T) {
        const int i = idx / n, l = idx - (idx / n) * n;
        A[i * lda + l] = 0.5 * (Hsub[((int64_t)c * nu + i) * nu + l] +
                                Hsub[((int64_t)c * nu + l) * nu + i]);
    }
    for (int idx = tid; idx < nr * n; idx += T) {
        const int r = idx / n, i = idx - (idx / n) * n;
        const double si = bscale[(int64_t)c * nu + i];
        double val;
        if (r == 0) {
            val = i == 0 ? 1.0 : 0.0;
        } else if (r == 1) {
            val = si * (double)Kc[(int64_t)i * m_pad + vpos(tinv, nb, c, jl)];
        } else if (r == npat + 2) {
            val = si * proj[(int64_t)c * nu + i];
        } else {
            const int atom = ci[kb + ((r - 2) >> 2)];
            const int64_t lr = Rg ? find_sorted(Rg, n_reg, atom) : atom;
            val = lr >= 0 ? si * (double)Kc[(int64_t)i * m_pad + vpos(tinv, nb, c, 4 * lr + ((r - 2) & 3))]
                          : 0.0;
        }
        R[r * lda + i] = val;
    }
    __syncthreads();
    // The stored basis K~ has unit S-norms and S-Gram matrix G = L L^T, so the
    // S-orthonormal basis K = K~ L^-T carries the subspace problem
    // A = L^-1 H~ L^-T and the rows q^T = q~^T L^-T and K_pat = K~_pat L^-T
    // (row 0, e_1^T, is unchanged: K^T S e_j = sqrt(S_jj) e_1).  Lsub holds
    // L^-1 (lower triangular); the products run in place from the last row
    // (column) down, which only reads rows (columns) not yet replaced.
    const double *Lc = Lsub + (int64_t)c * nu * nu;
    constexpr int kPer = (kMaxNu + kTriThreads - 1) / kTriThreads;   // entries per thread
    for (int i = n - 1; i >= 0; --i) {   // A <- L^-1 A, row i at a time
        const double *Li = Lc + (int64_t)i * nu;
        double x[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int col = tid + q * T;
            double s = 0.0;
            if (col < n)
                for (int m = 0; m <= i; ++m) s = fma(Li[m], A[m * lda + col], s);
            x[q] = s;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPer; ++q)
            if (tid + q * T < n) A[i * lda + tid + q * T] = x[q];
        __syncthreads();
    }
    // A <- A L^-T, column i at a time, rows i.. only: the result is symmetric
    // and from here on only its lower triangle (diagonal included) is read or
    // written.  Column i reads columns m <= i, which are not yet replaced, at
    // rows >= i.
    for (int i = n - 1; i >= 0; --i) {
        const double *Li = Lc + (int64_t)i * nu;
        double x[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int row = tid + q * T;
            double s = 0.0;
            if (row >= i && row < n)
                for (int m = 0; m <= i; ++m) s = fma(A[row * lda + m], Li[m], s);
            x[q] = s;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPer; ++q)
            if (tid + q * T >= i && tid + q * T < n) A[(tid + q * T) * lda + i] = x[q];
        __syncthreads();
    }
    for (int r = 1 + tid; r < nr; r += T) {   // R's rows 1..: R <- R L^-T, one row per thread
        double *x = R + r * lda;
        for (int i = n - 1; i >= 0; --i) {
            const double *Li = Lc + (int64_t)i * nu;
            double s = 0.0;
            for (int m = 0; m <= i; ++m) s = fma(x[m], Li[m], s);
            x[i] = s;
        }
    }
    __syncthreads();

    for (int k = 0; k + 2 < n; ++k) {
        const int L = n - k - 1;  // x = A[k+1 .. n-1][k]
        if (tid < 32) {
            double tail = 0.0;
            for (int l = 1 + tid; l < L; l += 32) {
                const double x = A[(k + 1 + l) * lda + k];
                tail += x * x;
            }
            tail = warp_sum(tail);
            if (tid == 0) {
                const double x0 = A[(k + 1) * lda + k];
                if (tail == 0.0) {
                    skip = 1;
                    ev[k] = x0;
                } else {
                    const double s = tail + x0 * x0;
                    const double alpha = -copysign(sqrt(s), x0);
                    const double v0 = x0 - alpha;
                    skip = 0;
                    ev[k] = alpha;
                    sc4[0] = 2.0 / (v0 * v0 + tail);   // reflector I - tau v v^T
                    sc4[1] = v0;
                }
            }
        }
        __syncthreads();
        if (skip) {
            __syncthreads();
            continue;
        }
        const double tauh = sc4[0];
        for (int l = tid; l < L; l += T) v[l] = (l == 0) ? sc4[1] : A[(k + 1 + l) * lda + k];
        __syncthreads();
        // p = tau A_sub v from A_sub's lower triangle, one entry per thread: row
        // col left of the diagonal (stride lda, odd, across the threads), then
        // column col from the diagonal down (consecutive addresses); p goes to
        // the scratch after e
        double *qv = ev + nu;
        double vp = 0.0;
        for (int col = tid; col < L; col += T) {
            const double *Ar = A + (k + 1 + col) * lda + (k + 1);
            double pl = 0.0;
            for (int m = 0; m < col; ++m) pl = fma(Ar[m], v[m], pl);
            for (int m = col; m < L; ++m) pl = fma(A[(k + 1 + m) * lda + (k + 1 + col)], v[m], pl);
            pl *= tauh;
            qv[col] = pl;
            vp = fma(v[col], pl, vp);
        }
        // K = (tau/2) v . p
        __shared__ double wpart[kTriThreads / 32];
        vp = warp_sum(vp);
        if ((tid & 31) == 0) wpart[tid >> 5] = vp;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int q = 0; q < T / 32; ++q) s += wpart[q];
            sc4[2] = 0.5 * tauh * s;
        }
        __syncthreads();
        for (int col = tid; col < L; col += T) qv[col] = fma(-sc4[2], v[col], qv[col]);   // q = p - K v
        __syncthreads();
        for (int idx = tid; idx < L * L; idx += T) {  // A_sub -= v q^T + q v^T, lower triangle
            const int a = idx / L, b = idx - (idx / L) * L;
            if (a >= b) A[(k + 1 + a) * lda + (k + 1 + b)] -= v[a] * qv[b] + qv[a] * v[b];
        }
        for (int r = tid; r < nr; r += T) {  // R <- R (I - tau v v^T) on columns k+1..
            double *row = R + r * lda + (k + 1);
            double s = 0.0;
            for (int m = 0; m < L; ++m) s = fma(row[m], v[m], s);
            s *= tauh;
            for (int m = 0; m < L; ++m) row[m] = fma(-s, v[m], row[m]);
        }
        __syncthreads();
    }
    double *Dc = D + (int64_t)sc * nu, *Ec = E + (int64_t)sc * nu;
    for (int i = tid; i < n; i += T) {
        Dc[i] = A[i * lda + i];
        Ec[i] = i + 2 < n ? ev[i] : (i + 2 == n ? A[(n - 1) * lda + (n - 2)] : 0.0);
    }
    double *RQc = RQ + (int64_t)sc * nr_max * nu;
    for (int idx = tid; idx < nr * n; idx += T) {
        const int r = idx / n, i = idx - (idx / n) * n;
        RQc[(int64_t)r * nu + i] = R[r * lda + i];
    }
}

// ------------------------------------------------------------------ batched QL
// Lane = subspace.  d and e live in shared memory as [i][lane].  Rotations go
// to rot[sc][0 .. rcap), sweeps (m, lo) to sweep[sc][0 .. scap); nsweep[sc]
// receives the sweep count, or -1 (no convergence in kQlMaxIter iterations for
// some level, or a full log).  Eigenvalues overwrite D, unsorted.
__global__ void __launch_bounds__(32) eig_ql_kernel(const int *__restrict__ bnu_eff, int cofs,
                                                    int nb, int nu, double *__restrict__ D,
                                                    const double *__restrict__ E,
                                                    double2 *__restrict__ rot, int64_t rcap,
                                                    int2 *__restrict__ sweep, int64_t scap,
                                                    int *__restrict__ nsweep)
{
    extern __shared__ __align__(16) double qsm[];
    const int lane = threadIdx.x;
    const int sc = blockIdx.x * 32 + lane;
    if (sc >= nb) return;
    double *d = qsm;                 // d[i] at d[i * 32 + lane]
    double *e = qsm + (size_t)nu * 32;
    const int n = bnu_eff[cofs + sc];
    for (int i = 0; i < n; ++i) {
        d[i * 32 + lane] = D[(int64_t)sc * nu + i];
        e[i * 32 + lane] = E[(int64_t)sc * nu + i];
    }
#define DD(i) d[(i) * 32 + lane]
#define EE(i) e[(i) * 32 + lane]
    double2 *rl = rot + (int64_t)sc * rcap;
    int2 *sl = sweep + (int64_t)sc * scap;
    int64_t nrot = 0;
    int nsw = 0;
    bool failed = false;
    for (int l = 0; l < n && !failed; ++l) {
        int iter = 0;
        while (true) {
            int m = l;
            for (; m < n - 1; ++m)
                if (fabs(EE(m)) <= DBL_EPSILON * (fabs(DD(m)) + fabs(DD(m + 1)))) break;
            if (m == l) break;
            if (++iter > kQlMaxIter || nrot + (m - l) > rcap || nsw >= scap) {
                failed = true;
                break;
            }
            double g = (DD(l + 1) - DD(l)) / (2.0 * EE(l));
            double r = hypot(g, 1.0);
            g = DD(m) - DD(l) + EE(l) / (g + copysign(r, g));
            double s = 1.0, cth = 1.0, p = 0.0;
            int i = m - 1;
            bool under = false;
            for (; i >= l; --i) {
                const double f = s * EE(i), b = cth * EE(i);
                // r = |(f, g)| as one square root and one reciprocal (the
                // levels and couplings are bounded by the spectrum's width, so
                // f^2 + g^2 neither overflows nor underflows to zero unless
                // both are zero)
                const double ss = fma(f, f, g * g);
                r = sqrt(ss);
                EE(i + 1) = r;
                if (r == 0.0) {
                    DD(i + 1) -= p;
                    EE(m) = 0.0;
                    under = true;
                    break;
                }
                const double rinv = 1.0 / r;
                s = f * rinv;
                cth = g * rinv;
                g = DD(i + 1) - p;
                r = (DD(i) - g) * s + 2.0 * cth * b;
                p = s * r;
                DD(i + 1) = g + p;
                g = cth * r - b;
                rl[nrot++] = make_double2(cth, s);
            }
            sl[nsw++] = make_int2(m, under ? i + 1 : l);
            if (!under) {
                DD(l) -= p;
                EE(l) = g;
                EE(m) = 0.0;
            }
        }
    }
    for (int i = 0; i < n; ++i) D[(int64_t)sc * nu + i] = DD(i);
    nsweep[sc] = failed ? -1 : nsw;
#undef DD
#undef EE
}

// ------------------------------------------------------------------ replay and outputs
__global__ void __launch_bounds__(kApplyThreads) eig_apply_kernel(
    const int *__restrict__ bnu_eff, const int *__restrict__ bstatus, int cofs, int nu,
    const int64_t *__restrict__ bcols, const double *__restrict__ sdiag,
    const int64_t *__restrict__ rp, int64_t col0, const double *__restrict__ D,
    const double *__restrict__ RQ, int nr_max, const double2 *__restrict__ rot, int64_t rcap,
    const int2 *__restrict__ sweep, int64_t scap, const int *__restrict__ nsweep,
    int *__restrict__ nu_eff_out, double *__restrict__ eps_out, double *__restrict__ w_out,
    double *__restrict__ t_out, double *__restrict__ P_out, const int64_t *__restrict__ p_off,
    int *__restrict__ eig_status, double *__restrict__ proj_out)
{
    const int sc = blockIdx.x;
    const int c = cofs + sc;
    const int64_t g = col0 + c;
    const int n = bnu_eff[c];
    const int tid = threadIdx.x, T = blockDim.x;
    const int ldr = nu | 1;
    extern __shared__ __align__(16) double asm_[];
    double *R = asm_;
    double *d = R + (size_t)nr_max * ldr;
    int *perm = reinterpret_cast<int *>(d + nu);
    const int64_t j = bcols[c];
    const int64_t J = j >> 2;
    const int npat = 4 * (int)(rp[J + 1] - rp[J]);
    const int nr = npat + 2 + (proj_out ? 1 : 0);
    const double *RQc = RQ + (int64_t)sc * nr_max * nu;
    for (int idx = tid; idx < nr * n; idx += T) {
        const int r = idx / n, i = idx - (idx / n) * n;
        R[r * ldr + i] = RQc[(int64_t)r * nu + i];
    }
    for (int i = tid; i < n; i += T) d[i] = D[(int64_t)sc * nu + i];
    __syncthreads();
    const int nsw = nsweep[sc];
    // each thread replays the whole log on its rows
    const double2 *rl = rot + (int64_t)sc * rcap;
    const int2 *sl = sweep + (int64_t)sc * scap;
    for (int r = tid; r < nr; r += T) {
        double *row = R + r * ldr;
        int64_t ptr = 0;
        for (int s = 0; s < nsw; ++s) {
            const int2 sw = sl[s];
            for (int i = sw.x - 1; i >= sw.y; --i) {
                const double2 cs = rl[ptr++];
                const double f = row[i + 1];
                row[i + 1] = fma(cs.y, row[i], cs.x * f);
                row[i] = fma(cs.x, row[i], -cs.y * f);
            }
        }
    }
    // rank of every level (ties by index): ascending order; a NaN level (from
    // non-finite input) ranks as +inf, so the ranks always form a permutation
    auto key = [&](int b) { const double x = d[b]; return x != x ? CUDART_INF : x; };
    for (int a = tid; a < n; a += T) {
        const double da = key(a);
        int rank = 0;
        for (int b = 0; b < n; ++b) {
            const double db = key(b);
            rank += (db < da) || (db == da && b < a);
        }
        perm[rank] = a;
    }
    __syncthreads();
    const double sq = sqrt(sdiag[j]);
    for (int a = tid; a < nu; a += T) {
        double ea = 0.0, wa = 0.0, ta = 0.0;
        if (a < n) {
            const int src = perm[a];
            ea = d[src];
            ta = R[1 * ldr + src];
            wa = sq * R[src] * ta;
        }
        eps_out[g * nu + a] = ea;
        t_out[g * nu + a] = ta;
        w_out[g * nu + a] = wa;
        if (proj_out) proj_out[g * nu + a] = a < n ? R[(npat + 2) * ldr + perm[a]] : 0.0;
    }
    double *P = P_out + p_off[g];
    for (int idx = tid; idx < npat * nu; idx += T) {
        const int r = idx / nu, a = idx - (idx / nu) * nu;
        P[idx] = a < n ? R[(r + 2) * ldr + perm[a]] : 0.0;
    }
    if (tid == 0) {
        nu_eff_out[g] = n;
        eig_status[g] = (nsw < 0 ? 1 : 0) | (bstatus[c] == 2 ? 2 : 0) | (bstatus[c] == 3 ? 4 : 0);
    }
}

template <typename VT>
cudaError_t tridiag_dispatch(const DeviceMatrix &A, const KrylovBatch &b, const RegionMaps *rm,
                             const EigScratch &es, int cofs, int nb2, cudaStream_t s)
{
    const int nu = b.nu;
    const size_t smem = eig_tridiag_smem(nu, es.nr_max, es.Ag != nullptr);
    cudaError_t e = allow_dynamic_smem((const void *)eig_tridiag_kernel<VT>, smem);
    if (e != cudaSuccess) return e;
    eig_tridiag_kernel<VT><<<nb2, kTriThreads, smem, s>>>(
        b.Hsub, b.nu_eff, b.scale, (const VT *)b.K, b.shape.m_pad, b.tinv, b.nb, nu, b.cols, A.rp, A.ci,
        rm ? rm->reg : nullptr, rm ? rm->n_reg : 0, cofs, es.D, es.E, es.RQ, es.nr_max, es.Ag, b.Lsub,
        es.proj);
    return cudaGetLastError();
}

}  // namespace

size_t eig_tridiag_smem(int nu, int nr_max, bool a_global)
{
    const size_t lda = (size_t)(nu | 1);
    return ((size_t)((a_global ? 0 : nu) + nr_max) * lda + 3 * (size_t)nu) * sizeof(double);
}

size_t eig_smem_bytes(int nu, int nr_max, bool a_global)
{
    const size_t lda = (size_t)(nu | 1);
    const size_t tri = eig_tridiag_smem(nu, nr_max, a_global);
    const size_t app = (size_t)nr_max * lda * sizeof(double) + (size_t)nu * (sizeof(double) + sizeof(int));
    const size_t ql = (size_t)2 * nu * 32 * sizeof(double);
    return std::max(tri, std::max(app, ql));
}

cudaError_t launch_eig(const DeviceMatrix &A, const KrylovBatch &b, const ColumnState &st,
                       int64_t col0, const RegionMaps *rm, const EigScratch &es, cudaStream_t s)
{
    if ((es.proj == nullptr) != (es.proj_out == nullptr)) return cudaErrorInvalidValue;
    const int nu = b.nu, ldr = nu | 1;
    const size_t qsmem = (size_t)2 * nu * 32 * sizeof(double);
    const size_t asmem = (size_t)es.nr_max * ldr * sizeof(double) + (size_t)nu * (sizeof(double) + sizeof(int));
    cudaError_t e;
    if ((e = allow_dynamic_smem((const void *)eig_ql_kernel, qsmem)) != cudaSuccess ||
        (e = allow_dynamic_smem((const void *)eig_apply_kernel, asmem)) != cudaSuccess)
        return e;
    for (int cofs = 0; cofs < b.nb; cofs += es.chunk) {
        const int nb2 = b.nb - cofs < es.chunk ? b.nb - cofs : es.chunk;
        e = b.prec == 0 ? tridiag_dispatch<double>(A, b, rm, es, cofs, nb2, s)
                        : tridiag_dispatch<float>(A, b, rm, es, cofs, nb2, s);
        if (e != cudaSuccess) return e;
        eig_ql_kernel<<<(nb2 + 31) / 32, 32, qsmem, s>>>(b.nu_eff, cofs, nb2, nu, es.D, es.E, es.rot,
                                                           es.rcap, es.sweep, es.scap, es.nsweep);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        eig_apply_kernel<<<nb2, kApplyThreads, asmem, s>>>(
            b.nu_eff, b.status, cofs, nu, b.cols, A.sdiag, A.rp, col0, es.D, es.RQ, es.nr_max,
            es.rot, es.rcap, es.sweep, es.scap, es.nsweep, st.nu_eff, st.eps, st.w, st.t, st.P,
            st.p_off, st.eig_status, es.proj ? es.proj_out : nullptr);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace marnoldi
