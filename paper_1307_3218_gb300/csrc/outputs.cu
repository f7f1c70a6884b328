// Fermi level and output columns of the multiple Arnoldi method on sm_103a.
//
// From each solved column's subspace levels eps_a, weights
// w_a = sqrt(S_jj) V[0][a] t_a and P_j = K_pat V (arXiv:1307.3218, Section 2:
// the Green's function determined by the subspace levels and vectors):
//   N(mu)       = sum_j sum_a 2 f w_a,   E = sum_j sum_a 2 f eps_a w_a
//   rho e_j     = P_j diag(2 f) t,   rho^E e_j = P_j diag(2 f eps) t
//   G(z) e_j    = P_j diag(1 / (z - eps)) t      (Eq. 1 inside L_nu^(j))
// with t = V^T K^T e_j and f(x) = 1 / (1 + e^x) at x = (eps - mu) / kT.
#include "internal.h"

namespace marnoldi {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double fermi(double x)
{
    if (x >= 0.0) {
        const double e = exp(-x);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + exp(x));
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
// them: each thread folds the partials q = tid, tid + blockDim.x, ... and the
// block reduces those in its fixed order.  No thread waits on another block.
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
    if (last) {   // uniform over the block
        __threadfence();
        const volatile double *vp = partial;
        double x = OP == 0 ? 0.0 : INFINITY, y = OP == 0 ? 0.0 : -INFINITY;
        for (unsigned q = threadIdx.x; q < gridDim.x; q += blockDim.x) {
            if (OP == 0) { x += vp[2 * q]; y += vp[2 * q + 1]; }
            else { x = fmin(x, vp[2 * q]); y = fmax(y, vp[2 * q + 1]); }
        }
        const double2 t = block_reduce2<OP>(x, y);
        if (threadIdx.x == 0) {
            out[0] = t.x;
            out[1] = t.y;
            *ticket = 0u;
        }
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

// Beyond |x| = 40 the Fermi function needs no exponential: for x < -40,
// 1 + e^x rounds to 1 in FP64, so f = 1 exactly; for x > 40, f < 4.3e-18 and
// is taken as 0 (each level's weight changes by less than 1e-17).
constexpr double kFermiCut = 40.0;

// Level-major order: element (a, c) = level a of column c, consecutive columns
// in consecutive lanes, so that the lanes of a warp hold levels at similar
// energies and mostly agree on whether the exponential is needed; levels
// a >= nu_eff[c] are skipped; the per-thread sums are reduced in a fixed
// order.  mu from mu_dev when given (the bisection graph), else mu_val.
__global__ void __launch_bounds__(256) count_kernel(int64_t ncols, int nu,
                                                    const int *__restrict__ nu_eff,
                                                    const double *__restrict__ eps,
                                                    const double *__restrict__ w, double mu_val,
                                                    const double *__restrict__ mu_dev, double kT,
                                                    double *partial, unsigned *ticket, double *out)
{
    const double mu = mu_dev ? *mu_dev : mu_val;
    const double cut = kFermiCut * kT;
    const int64_t total = ncols * nu, stride = (int64_t)gridDim.x * blockDim.x;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t a = idx / ncols, c = idx - a * ncols;
    const int64_t da = stride / ncols, dc = stride - da * ncols;
    double sn = 0.0, se = 0.0;
    for (; idx < total; idx += stride) {
        if (a < nu_eff[c]) {
            const double ea = eps[c * nu + a], d = ea - mu;
            const double f = d > cut ? 0.0 : (d < -cut ? 1.0 : fermi(d / kT));
            const double f2w = 2.0 * f * w[c * nu + a];
            sn += f2w;
            se = fma(f2w, ea, se);
        }
        a += da;
        c += dc;
        if (c >= ncols) {
            c -= ncols;
            ++a;
        }
    }
    finish_reduce<0>(sn, se, partial, ticket, out);
}

// One step of the Fermi-level bisection, run by one thread between two level
// counts inside the graph's while loop (same bracket, halving and stopping
// rule as a host loop would apply): phase 0 sets the bracket from the level
// range and asks for N(lo), phase 1 asks for N(hi), phase 2 checks that the
// bracket holds N_e, phase 3 halves until |N - N_e| <= rtol N_e or maxit
// halvings.  `steps` bounds the loop whatever the counts hold.
__global__ void bisect_step_kernel(BisectState *bs, const double *__restrict__ range,
                                   const double *__restrict__ out, double kT, double Ne,
                                   cudaGraphConditionalHandle loop)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    BisectState s = *bs;
    bool more = true;
    switch (s.phase) {
    case 0:
        // rounded like the host's (min - 40 kT): no contraction into an FMA
        s.lo = __dsub_rn(range[0], __dmul_rn(kBisectBracketKT, kT));
        s.hi = __dadd_rn(range[1], __dmul_rn(kBisectBracketKT, kT));
        s.mu = s.lo;
        s.phase = 1;
        break;
    case 1:
        s.Nlo = out[0];
        s.mu = s.hi;
        s.phase = 2;
        break;
    case 2:
        s.Nhi = out[0];
        if (!(s.Nlo <= Ne && Ne <= s.Nhi)) {
            s.status = 1;
            more = false;
        } else {
            s.it = 1;
            s.mu = 0.5 * (s.lo + s.hi);
            s.phase = 3;
        }
        break;
    case 3:
        s.N = out[0];
        s.E = out[1];
        if (fabs(s.N - Ne) <= kBisectRtol * Ne || s.it >= kBisectMaxit) {
            more = false;
        } else {
            if (s.N < Ne) s.lo = s.mu; else s.hi = s.mu;
            s.mu = 0.5 * (s.lo + s.hi);
            ++s.it;
        }
        break;
    default:
        more = false;
    }
    if (++s.steps >= kBisectMaxit + 3) more = false;
    if (!more) s.phase = 4;
    *bs = s;
    cudaGraphSetConditional(loop, more ? 1u : 0u);
}

// One CTA per solved column: y = 2 f t (and 2 f eps t), then the pattern rows
// P_j y written to block (I, J) entry [a][b] of the BSR output.
__global__ void __launch_bounds__(128) density_kernel(
    int nu, const int64_t *__restrict__ cols, const int *__restrict__ nu_eff,
    const double *__restrict__ eps, const double *__restrict__ t, const double *__restrict__ P,
    const int64_t *__restrict__ p_off, const int64_t *__restrict__ rp,
    const int64_t *__restrict__ tmap, double mu, double kT, double *__restrict__ rho,
    double *__restrict__ rhoE, int64_t nval)
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
        if (!in_range(o, nval, kChkDensityOut)) continue;
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

// Atomic forces from the density and energy-density matrices: one warp per
// atom K; lane l < 16 takes entry (a, b) = (l / 4, l % 4) of every block
// (K, J), J != K, with rho_bar = (rho_KJ + rho_JK^T) / 2 (k' = tmap[k] is the
// block (J, K)); F_K = 2 sum_J sum_ab (rho_bar dH - rho_bar^E dS), the lanes
// summed in a fixed order.  dH, dS: [3][nnzb][16], derivatives with respect
// to d = R_J - R_I.
__global__ void __launch_bounds__(256) force_kernel(int64_t nbr, int64_t nnzb, const int64_t *__restrict__ rp,
                                                    const int32_t *__restrict__ ci,
                                                    const int64_t *__restrict__ tmap,
                                                    const double *__restrict__ rho,
                                                    const double *__restrict__ rhoE,
                                                    const double *__restrict__ dH,
                                                    const double *__restrict__ dS, double *__restrict__ F)
{
    const int64_t K = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (K >= nbr) return;   // uniform over the warp
    double f[3] = {0.0, 0.0, 0.0};
    if (lane < 16) {
        const int lt = (lane & 3) * 4 + (lane >> 2);   // entry (b, a) of the mirror block
        for (int64_t k = rp[K]; k < rp[K + 1]; ++k) {
            if (ci[k] == K) continue;
            const int64_t kt = tmap[k];
            const double r = 0.5 * (rho[k * 16 + lane] + rho[kt * 16 + lt]);
            const double re = 0.5 * (rhoE[k * 16 + lane] + rhoE[kt * 16 + lt]);
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                const int64_t o = ((int64_t)x * nnzb + k) * 16 + lane;
                f[x] = fma(r, dH[o], fma(-re, dS[o], f[x]));
            }
        }
    }
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        double v = f[x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) F[3 * K + x] = 2.0 * v;
    }
}

}  // namespace

cudaError_t launch_forces(const DeviceMatrix &A, const double *rho, const double *rhoE, const double *dH,
                          const double *dS, double *F, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((A.nbr + 7) / 8);
    force_kernel<<<blocks, 256, 0, s>>>(A.nbr, A.nnzb, A.rp, A.ci, A.tmap, rho, rhoE, dH, dS, F);
    return cudaGetLastError();
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
    count_kernel<<<kReduceBlocks, 256, 0, s>>>(st.ncols, st.nu, st.nu_eff, st.eps, st.w, mu, nullptr,
                                                kT, partial, ticket, out);
    return cudaGetLastError();
}

cudaError_t launch_bisection(const ColumnState &st, double kT, double electron_count, double *partial,
                             unsigned *ticket, double *range, double *out, BisectState *bs,
                             cudaStream_t s)
{
    // the level range, then one graph whose while node alternates a bisection
    // step and a level count until the step clears the loop condition
    minmax_kernel<<<kReduceBlocks, 256, 0, s>>>(st.ncols * st.nu, st.nu, st.nu_eff, st.eps, partial,
                                                 ticket, range);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(bs, 0, sizeof(BisectState), s);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaStream_t cap = nullptr;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
    cudaGraphConditionalHandle loop;
    e = cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = loop;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    // the loop body, recorded from a private stream (capture mode local to
    // this thread, so other threads' CUDA calls are unaffected)
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            bisect_step_kernel<<<1, 32, 0, cap>>>(bs, range, out, kT, electron_count, loop);
            count_kernel<<<kReduceBlocks, 256, 0, cap>>>(st.ncols, st.nu, st.nu_eff, st.eps, st.w, 0.0,
                                                          &bs->mu, kT, partial, ticket, out);
            const cudaError_t el = cudaGetLastError();
            e = cudaStreamEndCapture(cap, &body);
            if (e == cudaSuccess) e = el;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ex, s);
    // destruction waits for nothing: launched work completes on its own
    if (ex) cudaGraphExecDestroy(ex);
    if (cap) cudaStreamDestroy(cap);
    cudaGraphDestroy(g);
    return e;
}

cudaError_t launch_density(const DeviceMatrix &A, const ColumnState &st, double mu, double kT,
                           double *rho, double *rhoE, cudaStream_t s)
{
    if (st.ncols == 0) return cudaSuccess;
    density_kernel<<<(unsigned)st.ncols, 128, 2 * st.nu * sizeof(double), s>>>(
        st.nu, st.cols, st.nu_eff, st.eps, st.t, st.P, st.p_off, A.rp, A.tmap, mu, kT, rho, rhoE, A.nnzb * 16);
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

MARNOLDI_CHECK_TAKE(outputs)

}  // namespace marnoldi
