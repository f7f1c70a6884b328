// Subspace eigensolve, Fermi level and output columns of the multiple Arnoldi
// method on sm_103a.
//
// Each subspace L_nu^(j) gives a nu x nu standard eigenproblem
// H_sub v_a = eps_a v_a whose levels and vectors determine the Green's
// function (arXiv:1307.3218, Section 2).  With q = K^T e_j and t = V^T q:
//   G(z) e_j    = K V diag(1 / (z - eps)) t        (Eq. 1 inside L_nu^(j))
//   rho e_j     = K V diag(2 f) t,   rho^E e_j = K V diag(2 f eps) t
//   N(mu)       = sum_j sum_a 2 f w_a,   E = sum_j sum_a 2 f eps_a w_a,
// with weights w_a = sqrt(S_jj) V[0][a] t_a (e_j^T S K = sqrt(S_jj) e_1^T) and
// f(x) = 1 / (1 + e^x) at x = (eps - mu) / kT.
//
// The eigensolver reduces H_sub to tridiagonal form with Householder
// reflections and diagonalises it with the implicit-shift QL algorithm
// (Bowdler, Martin, Reinsch & Wilkinson 1968).  One CTA owns one subspace:
// the reflections' matrix-vector and rank-2 updates are spread over the CTA;
// for QL, thread 0 runs each sweep's scalar recurrence and records its Givens
// rotations, then every thread applies them, in order, to its rows of the
// accumulated eigenvector matrix.  Only what the outputs need leaves the CTA:
// eps, w, t and P_j = K_pat V, the rows of K V on column j's pattern.
#include "internal.h"

#include <cfloat>

namespace marnoldi {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kEigThreads = 128;
constexpr int kQlMaxIter = 60;

__device__ __forceinline__ double warp_sum(double s)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    return s;
}

// Position of a in the ascending list R[0..n), or -1.
__device__ __forceinline__ int find_sorted(const int *__restrict__ R, int n, int a)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (R[mid] < a) lo = mid + 1; else hi = mid;
    }
    return (lo < n && R[lo] == a) ? lo : -1;
}

__device__ __forceinline__ double fermi(double x)
{
    if (x >= 0.0) {
        const double e = exp(-x);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + exp(x));
}

template <typename VT>
__global__ void __launch_bounds__(kEigThreads) eig_kernel(
    const double *__restrict__ Hsub, const int *__restrict__ bnu_eff,
    const int *__restrict__ bstatus, const double *__restrict__ bscale, const VT *__restrict__ K,
    int64_t m_pad, int nu, const int64_t *__restrict__ bcols,
    const double *__restrict__ sdiag, const int64_t *__restrict__ rp,
    const int32_t *__restrict__ ci, int64_t col0, int *__restrict__ nu_eff_out,
    double *__restrict__ eps_out, double *__restrict__ w_out, double *__restrict__ t_out,
    double *__restrict__ P_out, const int64_t *__restrict__ p_off, int *__restrict__ eig_status,
    const int *__restrict__ reg, int n_reg)
{
    const int c = blockIdx.x;
    const int64_t g = col0 + c;
    const int n = bnu_eff[c];
    const int tid = threadIdx.x, T = blockDim.x;
    extern __shared__ __align__(16) double sm[];
    double *A = sm;
    double *Q = A + nu * nu;
    double *d = Q + nu * nu;
    double *e = d + nu;
    double *vv = e + nu;
    double *pp = vv + nu;
    double *rc = pp + nu;
    double *rs = rc + nu;
    int *perm = reinterpret_cast<int *>(rs + nu);
    __shared__ double sc[4];
    __shared__ int si[4];

    for (int idx = tid; idx < n * n; idx += T) {
        const int i = idx / n, l = idx - (idx / n) * n;
        A[i * nu + l] = 0.5 * (Hsub[((int64_t)c * nu + i) * nu + l] +
                               Hsub[((int64_t)c * nu + l) * nu + i]);
        Q[i * nu + l] = (i == l) ? 1.0 : 0.0;
    }
    __syncthreads();

    // ---- Householder tridiagonalisation: A = Q T Q^T
    for (int k = 0; k + 2 < n; ++k) {
        const int L = n - k - 1;  // x = A[k+1 .. n-1][k]
        if (tid < 32) {
            double tail = 0.0;
            for (int l = 1 + tid; l < L; l += 32) {
                const double x = A[(k + 1 + l) * nu + k];
                tail += x * x;
            }
            tail = warp_sum(tail);
            if (tid == 0) {
                const double x0 = A[(k + 1) * nu + k];
                if (tail == 0.0) {
                    si[0] = 1;
                    e[k] = x0;
                } else {
                    const double s = tail + x0 * x0;
                    const double alpha = -copysign(sqrt(s), x0);
                    const double v0 = x0 - alpha;
                    si[0] = 0;
                    e[k] = alpha;
                    sc[0] = 2.0 / (v0 * v0 + tail);   // reflector I - tau v v^T
                    sc[1] = v0;
                }
            }
        }
        __syncthreads();
        if (si[0]) {
            __syncthreads();
            continue;
        }
        const double tauh = sc[0];
        for (int l = tid; l < L; l += T) vv[l] = (l == 0) ? sc[1] : A[(k + 1 + l) * nu + k];
        __syncthreads();
        for (int l = tid; l < L; l += T) {  // p = tau A_sub v
            const double *row = A + (k + 1 + l) * nu + (k + 1);
            double s = 0.0;
            for (int m = 0; m < L; ++m) s = fma(row[m], vv[m], s);
            pp[l] = tauh * s;
        }
        __syncthreads();
        if (tid < 32) {
            double s = 0.0;
            for (int l = tid; l < L; l += 32) s = fma(vv[l], pp[l], s);
            s = warp_sum(s);
            if (tid == 0) sc[2] = 0.5 * tauh * s;
        }
        __syncthreads();
        const double kc = sc[2];
        for (int l = tid; l < L; l += T) pp[l] = fma(-kc, vv[l], pp[l]);  // q = p - K v
        __syncthreads();
        for (int idx = tid; idx < L * L; idx += T) {  // A_sub -= v q^T + q v^T
            const int a = idx / L, b = idx - (idx / L) * L;
            A[(k + 1 + a) * nu + (k + 1 + b)] -= vv[a] * pp[b] + pp[a] * vv[b];
        }
        for (int i = tid; i < n; i += T) {  // Q <- Q (I - tau v v^T) on columns k+1..
            double *qrow = Q + i * nu + (k + 1);
            double s = 0.0;
            for (int m = 0; m < L; ++m) s = fma(qrow[m], vv[m], s);
            s *= tauh;
            for (int m = 0; m < L; ++m) qrow[m] = fma(-s, vv[m], qrow[m]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        for (int i = 0; i < n; ++i) d[i] = A[i * nu + i];
        if (n >= 2) e[n - 2] = A[(n - 1) * nu + (n - 2)];
        e[n - 1] = 0.0;
    }
    __syncthreads();

    // ---- implicit QL on (d, e); rotations accumulated into Q's columns
    int failed = 0;
    for (int l = 0; l < n && !failed; ++l) {
        int iter = 0;
        while (true) {
            if (tid == 0) {
                int m = l;
                for (; m < n - 1; ++m)
                    if (fabs(e[m]) <= DBL_EPSILON * (fabs(d[m]) + fabs(d[m + 1]))) break;
                if (m == l) {
                    si[1] = 0;
                } else if (iter >= kQlMaxIter) {
                    si[1] = -1;
                } else {
                    double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
                    double r = hypot(g, 1.0);
                    g = d[m] - d[l] + e[l] / (g + copysign(r, g));
                    double s = 1.0, cth = 1.0, p = 0.0;
                    int i = m - 1;
                    bool under = false;
                    for (; i >= l; --i) {
                        const double f = s * e[i], b = cth * e[i];
                        r = hypot(f, g);
                        e[i + 1] = r;
                        if (r == 0.0) {
                            d[i + 1] -= p;
                            e[m] = 0.0;
                            under = true;
                            break;
                        }
                        s = f / r;
                        cth = g / r;
                        g = d[i + 1] - p;
                        r = (d[i] - g) * s + 2.0 * cth * b;
                        p = s * r;
                        d[i + 1] = g + p;
                        g = cth * r - b;
                        rc[i] = cth;
                        rs[i] = s;
                    }
                    if (!under) {
                        d[l] -= p;
                        e[l] = g;
                        e[m] = 0.0;
                        si[2] = l;
                    } else {
                        si[2] = i + 1;
                    }
                    si[3] = m;
                    si[1] = 1;
                }
            }
            __syncthreads();
            const int flag = si[1], mm = si[3], lo = si[2];
            __syncthreads();
            if (flag <= 0) {
                failed = flag < 0;
                break;
            }
            for (int row = tid; row < n; row += T) {
                double *q = Q + row * nu;
                for (int i = mm - 1; i >= lo; --i) {
                    const double f = q[i + 1];
                    q[i + 1] = fma(rs[i], q[i], rc[i] * f);
                    q[i] = fma(rc[i], q[i], -rs[i] * f);
                }
            }
            __syncthreads();
            ++iter;
        }
    }
    if (tid == 0) eig_status[g] = (failed ? 1 : 0) | (bstatus[c] == 2 ? 2 : 0);

    // ---- ascending order; V = Q[:, perm] into A, sorted levels into pp
    if (tid == 0) {
        for (int a = 0; a < n; ++a) perm[a] = a;
        for (int a = 0; a < n; ++a) {
            int best = a;
            for (int b = a + 1; b < n; ++b)
                if (d[perm[b]] < d[perm[best]]) best = b;
            const int tmp = perm[a];
            perm[a] = perm[best];
            perm[best] = tmp;
        }
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += T) {
        const int i = idx / n, a = idx - (idx / n) * n;
        A[i * nu + a] = Q[i * nu + perm[a]];
    }
    for (int a = tid; a < n; a += T) pp[a] = d[perm[a]];
    // basis scales k_i = s_i w_i (e is free after QL); q = K^T e_j: entry jl of
    // every basis vector, jl = j in global mode, j's local index in a region
    const int64_t j = bcols[c];
    const int64_t J = j >> 2;
    const int *R = reg ? reg + (int64_t)c * n_reg : nullptr;
    const int pJ = R ? find_sorted(R, n_reg, (int)J) : 0;
    const int64_t jl = R ? 4 * (int64_t)(pJ < 0 ? 0 : pJ) + (j & 3) : j;
    const VT *Kc = K + (int64_t)c * nu * m_pad;
    for (int i = tid; i < n; i += T) {
        const double si = bscale[(int64_t)c * nu + i];
        e[i] = si;
        vv[i] = si * (double)Kc[(int64_t)i * m_pad + jl];
    }
    __syncthreads();
    const double sq = sqrt(sdiag[j]);
    for (int a = tid; a < nu; a += T) {
        double ta = 0.0, wa = 0.0, ea = 0.0;
        if (a < n) {
            for (int i = 0; i < n; ++i) ta = fma(A[i * nu + a], vv[i], ta);
            wa = sq * A[a] * ta;
            ea = pp[a];
        }
        eps_out[g * nu + a] = ea;
        t_out[g * nu + a] = ta;
        w_out[g * nu + a] = wa;
    }
    if (tid == 0) nu_eff_out[g] = n;
    // P_j = K_pat V on the 4 * (blocks of row j/4) pattern rows; in a region,
    // rows of atoms outside it are zero
    const int64_t kb = rp[J];
    const int npat = 4 * (int)(rp[J + 1] - kb);
    double *P = P_out + p_off[g];
    for (int idx = tid; idx < npat * nu; idx += T) {
        const int r = idx / nu, a = idx - (idx / nu) * nu;
        double s = 0.0;
        const int atom = ci[kb + (r >> 2)];
        const int64_t lr = R ? find_sorted(R, n_reg, atom) : atom;
        if (a < n && lr >= 0) {
            const int64_t row = 4 * lr + (r & 3);
            for (int i = 0; i < n; ++i)
                s = fma(e[i] * (double)Kc[(int64_t)i * m_pad + row], A[i * nu + a], s);
        }
        P[idx] = s;
    }
}

// Fixed-order block reduction of two values; thread 0 gets the totals.
template <int OP>  // 0 sum, 1 (min, max)
__device__ __forceinline__ double2 block_reduce2(double a, double b)
{
    __shared__ double2 red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ao = __shfl_xor_sync(kFull, a, o), bo = __shfl_xor_sync(kFull, b, o);
        if (OP == 0) { a += ao; b += bo; } else { a = fmin(a, ao); b = fmax(b, bo); }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) red[warp] = make_double2(a, b);
    __syncthreads();
    double2 r = red[0];
    if (threadIdx.x == 0)
        for (int q = 1; q < nw; ++q) {
            if (OP == 0) { r.x += red[q].x; r.y += red[q].y; }
            else { r.x = fmin(r.x, red[q].x); r.y = fmax(r.y, red[q].y); }
        }
    return r;
}

// Per-block partials, then the last block to finish (atomic ticket) combines
// them in block order; no thread waits on another block.
template <int OP>
__device__ void finish_reduce(double a, double b, double *partial, unsigned *ticket, double *out)
{
    __shared__ int last;
    const double2 r = block_reduce2<OP>(a, b);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = r.x;
        partial[2 * blockIdx.x + 1] = r.y;
        __threadfence();
        last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const volatile double *vp = partial;
        double x = vp[0], y = vp[1];
        for (unsigned q = 1; q < gridDim.x; ++q) {
            if (OP == 0) { x += vp[2 * q]; y += vp[2 * q + 1]; }
            else { x = fmin(x, vp[2 * q]); y = fmax(y, vp[2 * q + 1]); }
        }
        out[0] = x;
        out[1] = y;
        *ticket = 0u;
    }
}

__global__ void __launch_bounds__(256) minmax_kernel(int64_t total, int nu,
                                                     const int *__restrict__ nu_eff,
                                                     const double *__restrict__ eps,
                                                     double *partial, unsigned *ticket, double *out)
{
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = idx / nu;
        if (idx - c * nu < nu_eff[c]) {
            lo = fmin(lo, eps[idx]);
            hi = fmax(hi, eps[idx]);
        }
    }
    finish_reduce<1>(lo, hi, partial, ticket, out);
}

__global__ void __launch_bounds__(256) count_kernel(int64_t total, int nu,
                                                    const int *__restrict__ nu_eff,
                                                    const double *__restrict__ eps,
                                                    const double *__restrict__ w, double mu,
                                                    double kT, double *partial, unsigned *ticket,
                                                    double *out)
{
    double sn = 0.0, se = 0.0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = idx / nu;
        if (idx - c * nu < nu_eff[c]) {
            const double ea = eps[idx];
            const double f2w = 2.0 * fermi((ea - mu) / kT) * w[idx];
            sn += f2w;
            se = fma(f2w, ea, se);
        }
    }
    finish_reduce<0>(sn, se, partial, ticket, out);
}

// One CTA per solved column: y = 2 f t (and 2 f eps t), then the pattern rows
// P_j y written to block (I, J) entry [a][b] of the BSR output.
__global__ void __launch_bounds__(128) density_kernel(
    int nu, const int64_t *__restrict__ cols, const int *__restrict__ nu_eff,
    const double *__restrict__ eps, const double *__restrict__ t, const double *__restrict__ P,
    const int64_t *__restrict__ p_off, const int64_t *__restrict__ rp,
    const int64_t *__restrict__ tmap, double mu, double kT, double *__restrict__ rho,
    double *__restrict__ rhoE)
{
    extern __shared__ double ys[];
    double *y = ys, *ye = ys + nu;
    const int64_t c = blockIdx.x;
    const int64_t j = cols[c], J = j >> 2;
    const int b = (int)(j & 3), n = nu_eff[c];
    for (int a = threadIdx.x; a < nu; a += blockDim.x) {
        double v = 0.0, ve = 0.0;
        if (a < n) {
            const double ea = eps[c * nu + a];
            const double f2t = 2.0 * fermi((ea - mu) / kT) * t[c * nu + a];
            v = f2t;
            ve = f2t * ea;
        }
        y[a] = v;
        ye[a] = ve;
    }
    __syncthreads();
    const int64_t kb = rp[J];
    const int npat = 4 * (int)(rp[J + 1] - kb);
    const double *Pc = P + p_off[c];
    for (int r = threadIdx.x; r < npat; r += blockDim.x) {
        double s = 0.0, se = 0.0;
        const double *row = Pc + (int64_t)r * nu;
        for (int a = 0; a < n; ++a) {
            s = fma(row[a], y[a], s);
            se = fma(row[a], ye[a], se);
        }
        const int64_t o = tmap[kb + (r >> 2)] * 16 + (r & 3) * 4 + b;
        rho[o] = s;
        rhoE[o] = se;
    }
}

__global__ void __launch_bounds__(128) green_kernel(
    int nu, const int64_t *__restrict__ cols, const int *__restrict__ nu_eff,
    const double *__restrict__ eps, const double *__restrict__ t, const double *__restrict__ P,
    const int64_t *__restrict__ p_off, const int64_t *__restrict__ rp,
    const int64_t *__restrict__ tmap, double zr, double zi, double *__restrict__ G)
{
    extern __shared__ double ys[];
    double *yr = ys, *yi = ys + nu;
    const int64_t c = blockIdx.x;
    const int64_t j = cols[c], J = j >> 2;
    const int b = (int)(j & 3), n = nu_eff[c];
    for (int a = threadIdx.x; a < nu; a += blockDim.x) {
        double vr = 0.0, vi = 0.0;
        if (a < n) {  // t / (z - eps) = t (conj(z) - eps) / |z - eps|^2
            const double dr = zr - eps[c * nu + a];
            const double den = dr * dr + zi * zi;
            const double ta = t[c * nu + a];
            vr = ta * dr / den;
            vi = -ta * zi / den;
        }
        yr[a] = vr;
        yi[a] = vi;
    }
    __syncthreads();
    const int64_t kb = rp[J];
    const int npat = 4 * (int)(rp[J + 1] - kb);
    const double *Pc = P + p_off[c];
    for (int r = threadIdx.x; r < npat; r += blockDim.x) {
        double sr = 0.0, sim = 0.0;
        const double *row = Pc + (int64_t)r * nu;
        for (int a = 0; a < n; ++a) {
            sr = fma(row[a], yr[a], sr);
            sim = fma(row[a], yi[a], sim);
        }
        const int64_t o = tmap[kb + (r >> 2)] * 16 + (r & 3) * 4 + b;
        G[2 * o] = sr;
        G[2 * o + 1] = sim;
    }
}

template <typename VT>
cudaError_t eig_dispatch(const DeviceMatrix &A, const KrylovBatch &b, const ColumnState &st,
                         int64_t col0, const RegionMaps *rm, cudaStream_t s)
{
    const int nu = b.nu;
    const size_t smem = (size_t)(2 * nu * nu + 6 * nu) * sizeof(double) + (size_t)nu * sizeof(int);
    static bool configured = false;
    if (!configured) {
        const size_t maxs = (size_t)(2 * kMaxNu * kMaxNu + 6 * kMaxNu) * sizeof(double) +
                            (size_t)kMaxNu * sizeof(int);
        cudaError_t e = cudaFuncSetAttribute(eig_kernel<VT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)maxs);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    eig_kernel<VT><<<b.nb, kEigThreads, smem, s>>>(
        b.Hsub, b.nu_eff, b.status, b.scale, (const VT *)b.K, b.shape.m_pad, nu, b.cols, A.sdiag, A.rp, A.ci, col0,
        st.nu_eff, st.eps, st.w, st.t, st.P, st.p_off, st.eig_status, rm ? rm->reg : nullptr,
        rm ? rm->n_reg : 0);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_eig(const DeviceMatrix &A, const KrylovBatch &b, const ColumnState &st,
                       int64_t col0, const RegionMaps *rm, cudaStream_t s)
{
    return b.prec == 0 ? eig_dispatch<double>(A, b, st, col0, rm, s)
                       : eig_dispatch<float>(A, b, st, col0, rm, s);
}

cudaError_t launch_minmax(const ColumnState &st, double *partial, unsigned *ticket, double *out,
                          cudaStream_t s)
{
    minmax_kernel<<<kReduceBlocks, 256, 0, s>>>(st.ncols * st.nu, st.nu, st.nu_eff, st.eps,
                                                 partial, ticket, out);
    return cudaGetLastError();
}

cudaError_t launch_count(const ColumnState &st, double mu, double kT, double *partial,
                         unsigned *ticket, double *out, cudaStream_t s)
{
    count_kernel<<<kReduceBlocks, 256, 0, s>>>(st.ncols * st.nu, st.nu, st.nu_eff, st.eps, st.w,
                                                mu, kT, partial, ticket, out);
    return cudaGetLastError();
}

cudaError_t launch_density(const DeviceMatrix &A, const ColumnState &st, double mu, double kT,
                           double *rho, double *rhoE, cudaStream_t s)
{
    if (st.ncols == 0) return cudaSuccess;
    density_kernel<<<(unsigned)st.ncols, 128, 2 * st.nu * sizeof(double), s>>>(
        st.nu, st.cols, st.nu_eff, st.eps, st.t, st.P, st.p_off, A.rp, A.tmap, mu, kT, rho, rhoE);
    return cudaGetLastError();
}

cudaError_t launch_green(const DeviceMatrix &A, const ColumnState &st, double zr, double zi,
                         double *G, cudaStream_t s)
{
    if (st.ncols == 0) return cudaSuccess;
    green_kernel<<<(unsigned)st.ncols, 128, 2 * st.nu * sizeof(double), s>>>(
        st.nu, st.cols, st.nu_eff, st.eps, st.t, st.P, st.p_off, A.rp, A.tmap, zr, zi, G);
    return cudaGetLastError();
}

}  // namespace marnoldi
