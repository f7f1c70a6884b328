// The k-th eigen level and vector from the subspace levels and vectors of the
// multiple Arnoldi method (arXiv:1307.3218, Section 2, the paragraph on the
// k-th eigen level and Eq. 3; the sign rule of its Appendix).
//
// With the smoothed step theta(eta - eps) = f((eps - eta) / sigma) the
// integrated density of states is n(eta) = sum_j sum_a w_a f((eps_a - eta) /
// sigma) (the level count's reduction without the spin factor), eta(n) its
// inverse, eps_k = eta(k - 1/2), and component j of phi_k is
// sum_a s_a t_a W_a with W_a = theta(eta(k) - eps_a) - theta(eta(k-1) - eps_a)
// and t_a = e_j^T K v_a.  The signs s_a = sign(v_ref^T K v_a) come from a
// reference subspace eigenvector v_ref (the one of largest |t_a W_a|).
//
//   window_kernel   per column: the largest |t_a W_a| and its level
//   argmax_kernel   one CTA: the column and level of the largest (first among equals)
//   eigvec_kernel   one CTA: the full-space vector K v_a of one level of one
//                   column of the current batch (inverse iteration on the
//                   nu x nu problem, then a sum over the stored vectors)
//   project_kernel  per batch column: v^T w_i for every stored vector
//                   (the extra row the eigensolver turns into v^T K v_a)
//   combine_kernel  per solved column: component j of phi_k with the signs
#include "internal.h"

namespace marnoldi {
namespace {

__device__ __forceinline__ double step_f(double x)   // f(x) = 1 / (1 + e^x), x may be +-inf
{
    if (x >= 0.0) {
        const double e = exp(-x);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + exp(x));
}

__device__ __forceinline__ double window(double eps, double lo, double hi, double sigma)
{
    return step_f((eps - hi) / sigma) - step_f((eps - lo) / sigma);
}

__global__ void __launch_bounds__(256) window_kernel(int64_t ncols, int nu, const int *__restrict__ nu_eff,
                                                     const double *__restrict__ eps,
                                                     const double *__restrict__ t, double lo, double hi,
                                                     double sigma, double *__restrict__ colmax,
                                                     int *__restrict__ colarg)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    double best = -1.0;
    int arg = 0;
    for (int a = 0; a < nu_eff[c]; ++a) {
        const double v = fabs(t[c * nu + a] * window(eps[c * nu + a], lo, hi, sigma));
        if (v > best) {
            best = v;
            arg = a;
        }
    }
    colmax[c] = best < 0.0 ? 0.0 : best;
    colarg[c] = arg;
}

__global__ void __launch_bounds__(1024) argmax_kernel(int64_t ncols, const double *__restrict__ colmax,
                                                      int64_t *__restrict__ out)
{
    __shared__ double bv[1024];
    __shared__ int64_t bi[1024];
    double v = -1.0;
    int64_t i = -1;
    for (int64_t c = threadIdx.x; c < ncols; c += blockDim.x)
        if (colmax[c] > v) {
            v = colmax[c];
            i = c;
        }
    bv[threadIdx.x] = v;
    bi[threadIdx.x] = i;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double v2 = bv[threadIdx.x + s];
            const int64_t i2 = bi[threadIdx.x + s];
            if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 >= 0 && (bi[threadIdx.x] < 0 || i2 < bi[threadIdx.x]))) {
                bv[threadIdx.x] = v2;
                bi[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = bi[0];
}

// position -> tile of batch column c (positions of the tiles in use)
__device__ void inverse_tiles(const uint16_t *__restrict__ tinv, int nb, int c, int ntile, int npos,
                              int *__restrict__ inv)
{
    for (int p = threadIdx.x; p < npos; p += blockDim.x) inv[p] = -1;
    __syncthreads();
    for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
        const int p = tinv[(int64_t)t * nb + c];
        if (p < npos) inv[p] = t;
    }
    __syncthreads();
}

// fixed-order sum over the CTA (256 threads); every thread gets the total
__device__ double cta_sum(double x, double *red)
{
    red[threadIdx.x] = x;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double total = red[0];
    __syncthreads();
    return total;
}

template <typename VT>
__global__ void __launch_bounds__(256) project_kernel(const VT *__restrict__ K, const int *__restrict__ nu_eff,
                                                      const uint16_t *__restrict__ tinv,
                                                      const int *__restrict__ tcnt, int nb, int ntile,
                                                      int nu, int64_t m_pad, int64_t M,
                                                      const double *__restrict__ v, double *__restrict__ proj)
{
    __shared__ int inv[kMaxTiles];
    __shared__ double red[256];
    const int c = blockIdx.x;
    const int npos = (int)(m_pad / 32);
    inverse_tiles(tinv, nb, c, ntile, npos, inv);
    const int n = nu_eff[c];
    for (int i = 0; i < nu; ++i) {
        double s = 0.0;
        if (i < n) {
            const int64_t len = 32 * (int64_t)tcnt[(int64_t)c * (nu + 2) + i];
            const VT *w = K + ((int64_t)c * nu + i) * m_pad;
            for (int64_t p = threadIdx.x; p < len; p += blockDim.x) {
                const int t = inv[p >> 5];
                const int64_t r = 32 * (int64_t)t + (p & 31);
                if (t >= 0 && r < M) s = fma((double)w[p], v[r], s);
            }
        }
        const double total = cta_sum(s, red);
        if (threadIdx.x == 0) proj[(int64_t)c * nu + i] = total;
    }
}

// The vector K v_a of batch column c for the level eps: A = L^-1 H~ L^-T as
// in the eigensolve, two steps of inverse iteration on A - (eps + delta) I
// with partial-pivoting LU, y = L^-T v, then
// out[r] = sum_i s_i y_i w_i[pos(r)] over the rows in the column's tiles.
// A sits in shared memory up to n = kSmemEigvec, else in the global scratch Ag
// (n <= kMaxNu; one CTA, so it stays in L2).
constexpr int kSmemEigvec = 128;

template <typename VT>
__global__ void __launch_bounds__(256) eigvec_kernel(
    int c, double eps, const double *__restrict__ Hsub, const double *__restrict__ Lsub,
    const double *__restrict__ scale, const int *__restrict__ nu_eff, const VT *__restrict__ K,
    const uint16_t *__restrict__ tinv, int nb, int ntile, int nu, int64_t m_pad, int64_t M,
    double *__restrict__ out, double *__restrict__ Ag)
{
    extern __shared__ __align__(16) double es[];
    __shared__ int inv[kMaxTiles];
    __shared__ int piv[kMaxNu];
    __shared__ double x[kMaxNu], y[kMaxNu];
    const int n = nu_eff[c];
    const int lda = n | 1;
    double *A = Ag ? Ag : es;
    const int tid = threadIdx.x, T = blockDim.x;
    const double *Lc = Lsub + (int64_t)c * nu * nu;
    for (int idx = tid; idx < n * n; idx += T) {
        const int i = idx / n, l = idx - i * n;
        A[i * lda + l] = 0.5 * (Hsub[((int64_t)c * nu + i) * nu + l] + Hsub[((int64_t)c * nu + l) * nu + i]);
    }
    __syncthreads();
    for (int i = n - 1; i >= 0; --i) {   // A <- L^-1 A, row i from rows <= i
        double v[kMaxNu / 256 + 1];
        for (int q = 0; q * T + tid < n; ++q) {
            const int col = q * T + tid;
            double s = 0.0;
            for (int m = 0; m <= i; ++m) s = fma(Lc[(int64_t)i * nu + m], A[m * lda + col], s);
            v[q] = s;
        }
        __syncthreads();
        for (int q = 0; q * T + tid < n; ++q) A[i * lda + q * T + tid] = v[q];
        __syncthreads();
    }
    for (int i = n - 1; i >= 0; --i) {   // A <- A L^-T, column i from columns <= i
        double v[kMaxNu / 256 + 1];
        for (int q = 0; q * T + tid < n; ++q) {
            const int row = q * T + tid;
            double s = 0.0;
            for (int m = 0; m <= i; ++m) s = fma(A[row * lda + m], Lc[(int64_t)i * nu + m], s);
            v[q] = s;
        }
        __syncthreads();
        for (int q = 0; q * T + tid < n; ++q) A[(q * T + tid) * lda + i] = v[q];
        __syncthreads();
    }
    // shift just off the level, so that the solve stays regular while the
    // level's direction dominates the solution
    const double shift = eps + 1e-10 * fmax(1.0, fabs(eps));
    for (int i = tid; i < n; i += T) A[i * lda + i] -= shift;
    __syncthreads();
    for (int k = 0; k < n; ++k) {   // LU with partial pivoting
        if (tid == 0) {
            int p = k;
            double best = fabs(A[k * lda + k]);
            for (int r = k + 1; r < n; ++r)
                if (fabs(A[r * lda + k]) > best) {
                    best = fabs(A[r * lda + k]);
                    p = r;
                }
            piv[k] = p;
            if (A[p * lda + k] == 0.0) A[p * lda + k] = 1e-300;   // exactly singular: any direction
        }
        __syncthreads();
        const int p = piv[k];
        if (p != k)
            for (int col = tid; col < n; col += T) {
                const double a = A[k * lda + col];
                A[k * lda + col] = A[p * lda + col];
                A[p * lda + col] = a;
            }
        __syncthreads();
        const double inv_p = 1.0 / A[k * lda + k];
        for (int r = k + 1 + tid; r < n; r += T) A[r * lda + k] *= inv_p;
        __syncthreads();
        const int m = n - k - 1;
        for (int idx = tid; idx < m * m; idx += T) {
            const int r = k + 1 + idx / m, col = k + 1 + idx % m;
            A[r * lda + col] = fma(-A[r * lda + k], A[k * lda + col], A[r * lda + col]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        for (int i = 0; i < n; ++i) x[i] = 1.0;
        for (int it = 0; it < 2; ++it) {
            for (int k = 0; k < n; ++k) {   // b <- P b
                const double a = x[k];
                x[k] = x[piv[k]];
                x[piv[k]] = a;
            }
            for (int i = 0; i < n; ++i)     // L (unit lower)
                for (int m = 0; m < i; ++m) x[i] = fma(-A[i * lda + m], x[m], x[i]);
            for (int i = n - 1; i >= 0; --i) {   // U
                for (int m = i + 1; m < n; ++m) x[i] = fma(-A[i * lda + m], x[m], x[i]);
                x[i] /= A[i * lda + i];
            }
            double nrm = 0.0;
            for (int i = 0; i < n; ++i) nrm = fma(x[i], x[i], nrm);
            nrm = sqrt(nrm);
            for (int i = 0; i < n; ++i) x[i] /= nrm;
        }
    }
    __syncthreads();
    for (int i = tid; i < n; i += T) {   // y = L^-T v, times the stored vectors' scales
        double s = 0.0;
        for (int m = i; m < n; ++m) s = fma(Lc[(int64_t)m * nu + i], x[m], s);
        y[i] = s * scale[(int64_t)c * nu + i];
    }
    const int npos = (int)(m_pad / 32);
    inverse_tiles(tinv, nb, c, ntile, npos, inv);
    const VT *Kc = K + (int64_t)c * nu * m_pad;
    for (int64_t p = tid; p < m_pad; p += T) {
        const int t = inv[p >> 5];
        const int64_t r = 32 * (int64_t)t + (p & 31);
        if (t < 0 || r >= M) continue;
        double s = 0.0;
        for (int i = 0; i < n; ++i) s = fma(y[i], (double)Kc[(int64_t)i * m_pad + p], s);
        out[r] = s;
    }
}

__global__ void __launch_bounds__(256) combine_kernel(int64_t ncols, int nu, const int64_t *__restrict__ cols,
                                                      const int *__restrict__ nu_eff,
                                                      const double *__restrict__ eps,
                                                      const double *__restrict__ t,
                                                      const double *__restrict__ proj, double lo, double hi,
                                                      double sigma, double *__restrict__ phi)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    double s = 0.0;
    for (int a = 0; a < nu_eff[c]; ++a) {
        const double sg = proj[c * nu + a] < 0.0 ? -1.0 : 1.0;
        s = fma(sg * t[c * nu + a], window(eps[c * nu + a], lo, hi, sigma), s);
    }
    phi[cols[c]] = s;
}

}  // namespace

cudaError_t launch_window(const ColumnState &st, double lo, double hi, double sigma, double *colmax, int *colarg,
                          int64_t *argmax, cudaStream_t s)
{
    if (st.ncols < 1) return cudaErrorInvalidValue;
    window_kernel<<<(unsigned)((st.ncols + 255) / 256), 256, 0, s>>>(st.ncols, st.nu, st.nu_eff, st.eps, st.t, lo,
                                                                     hi, sigma, colmax, colarg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    argmax_kernel<<<1, 1024, 0, s>>>(st.ncols, colmax, argmax);
    return cudaGetLastError();
}

cudaError_t launch_project(const KrylovBatch &b, const double *v, int64_t M, double *proj, cudaStream_t s)
{
    if (b.ntile > kMaxTiles) return cudaErrorInvalidValue;
    if (b.prec == 0)
        project_kernel<double><<<b.nb, 256, 0, s>>>((const double *)b.K, b.nu_eff, b.tinv, b.tcnt, b.nb, b.ntile,
                                                    b.nu, b.shape.m_pad, M, v, proj);
    else
        project_kernel<float><<<b.nb, 256, 0, s>>>((const float *)b.K, b.nu_eff, b.tinv, b.tcnt, b.nb, b.ntile,
                                                   b.nu, b.shape.m_pad, M, v, proj);
    return cudaGetLastError();
}

int eigvec_max_nu() { return kMaxNu; }

size_t eigvec_scratch_bytes(int nu) { return nu > kSmemEigvec ? (size_t)nu * (nu | 1) * sizeof(double) : 0; }

cudaError_t launch_eigvec(const KrylovBatch &b, int c, double eps, int64_t M, double *out, double *Ag,
                          cudaStream_t s)
{
    if (b.nu > kMaxNu || c < 0 || c >= b.nb || b.ntile > kMaxTiles) return cudaErrorInvalidValue;
    if (b.nu > kSmemEigvec && !Ag) return cudaErrorInvalidValue;
    const bool in_smem = b.nu <= kSmemEigvec;
    const size_t smem = in_smem ? (size_t)kSmemEigvec * (kSmemEigvec | 1) * sizeof(double) : 0;
    double *ag = in_smem ? nullptr : Ag;
    cudaError_t e;
    if (b.prec == 0) {
        if ((e = allow_dynamic_smem((const void *)eigvec_kernel<double>, smem)) != cudaSuccess) return e;
        eigvec_kernel<double><<<1, 256, smem, s>>>(c, eps, b.Hsub, b.Lsub, b.scale, b.nu_eff, (const double *)b.K,
                                                   b.tinv, b.nb, b.ntile, b.nu, b.shape.m_pad, M, out, ag);
    } else {
        if ((e = allow_dynamic_smem((const void *)eigvec_kernel<float>, smem)) != cudaSuccess) return e;
        eigvec_kernel<float><<<1, 256, smem, s>>>(c, eps, b.Hsub, b.Lsub, b.scale, b.nu_eff, (const float *)b.K,
                                                  b.tinv, b.nb, b.ntile, b.nu, b.shape.m_pad, M, out, ag);
    }
    return cudaGetLastError();
}

cudaError_t launch_combine(const ColumnState &st, const double *proj, double lo, double hi, double sigma,
                           double *phi, cudaStream_t s)
{
    if (st.ncols < 1) return cudaSuccess;
    combine_kernel<<<(unsigned)((st.ncols + 255) / 256), 256, 0, s>>>(st.ncols, st.nu, st.cols, st.nu_eff, st.eps,
                                                                      st.t, proj, lo, hi, sigma, phi);
    return cudaGetLastError();
}

}  // namespace marnoldi
