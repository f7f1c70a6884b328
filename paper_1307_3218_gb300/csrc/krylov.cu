// Krylov-subspace build of the multiple Arnoldi method on sm_103a.
//
// For a batch of columns j, builds the S-orthonormal basis K of
// span{e_j, H e_j, ..., H^(nu-1) e_j} (arXiv:1307.3218, Section 2: the subspace
// L_nu^(j) containing e_j whose nu x nu *standard* eigenproblem replaces
// H phi = eps S phi, Eq. 2) and the explicit subspace matrix H_sub = K^T H K.
//
// One Krylov step n, for every column of the batch:
//   spmm(H):    u = H k_n                                (BSR 4x4 x batch panel)
//   mgs:        h_{i,n} = k_i . u (i <= n), then two passes of modified
//               Gram-Schmidt in the S inner product using the stored S k_i:
//               c_i = (S k_i) . w, w -= c_i k_i
//   spmm(S):    S w
//   normalize:  beta = sqrt(w . S w), k_{n+1} = w / beta, S k_{n+1} = S w / beta,
//               or stop the column when beta^2 <= tau^2 (beta^2 + sum_i c_i^2),
//               i.e. ||w||_S <= tau ||u||_S (S-orthogonality of K splits
//               ||u||_S^2 into beta^2 plus the squared projection coefficients).
//
// Inner products are always accumulated in FP64; in mixed precision the
// vectors, the SpMM and the Gram-Schmidt updates are FP32.  Reductions use a
// fixed order (warp butterfly, then warps in index order), so results do not
// depend on scheduling.
#include "internal.h"

#include <cstdio>

namespace marnoldi {

const char *kernel_name(int kind)
{
    static const char *names[KK_NKINDS] = {"init",   "spmm_H",  "mgs",   "spmm_S",  "normalize",
                                           "eigsub", "minmax",  "count", "density", "green"};
    return (kind >= 0 && kind < KK_NKINDS) ? names[kind] : "?";
}

ColumnShape column_shape(int64_t m)
{
    ColumnShape s{1, 32, 32};
    for (int v = 1; v <= 16; v *= 2) {
        int64_t t = (m + v - 1) / v;
        if (t <= 1024 || v == 16) {
            t = v >= 8 ? 1024 : ((t + 31) / 32) * 32;   // vpt >= 8: T fixed at compile time
            s.vpt = v;
            s.threads = (int)t;
            s.m_pad = t * v;
            break;
        }
    }
    return s;
}

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ dot accumulators
// Per-thread partial inner products.  FP64 vectors: fused multiply-adds in
// FP64.  FP32 vectors (mixed precision): the product a*b of two floats is
// split exactly into p + e (p = fl(a*b), e = fma(a, b, -p)) and p is added to
// the running sum with an exact two-sum, so the pair (hi, lo) carries the sum
// to about 2^-48 relative.  The reduction across the CTA stays in such pairs
// and only the CTA total is converted to FP64, so the inner products are
// FP64-accurate on FP32 data with no per-element FP64 work (GB300 issues
// FP32 at about 64 times its FP64 rate).  The _rn intrinsics keep the
// compiler from contracting the error-free steps into FMAs.
__device__ __forceinline__ void df_add(float &hi, float &lo, float h2, float l2)
{
    const float s = __fadd_rn(hi, h2);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(l2, err));
}

template <typename VT> struct DotAcc;
template <> struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
    __device__ __forceinline__ void warp_reduce()
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    }
    __device__ __forceinline__ static double2 pack(const DotAcc &a, const DotAcc &b)
    {
        return make_double2(a.s, b.s);
    }
    __device__ __forceinline__ static void unpack(double2 p, DotAcc &a, DotAcc &b)
    {
        a.s = p.x;
        b.s = p.y;
    }
};
template <> struct DotAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        df_add(hi, lo, p, e);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
    __device__ __forceinline__ void warp_reduce()
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(kFull, hi, o);
            const float l2 = __shfl_xor_sync(kFull, lo, o);
            df_add(hi, lo, h2, l2);
        }
    }
    __device__ __forceinline__ static double2 pack(const DotAcc &a, const DotAcc &b)
    {
        union { float4 f; double2 d; } u;
        u.f = make_float4(a.hi, a.lo, b.hi, b.lo);
        return u.d;
    }
    __device__ __forceinline__ static void unpack(double2 p, DotAcc &a, DotAcc &b)
    {
        union { float4 f; double2 d; } u;
        u.d = p;
        a.hi = u.f.x; a.lo = u.f.y; b.hi = u.f.z; b.lo = u.f.w;
    }
};

// Sum of two per-thread accumulators over the CTA, in a fixed order (warp
// butterflies, then warp 0 over the warps' partials); every thread returns
// the same FP64 totals.  Only warp 0 touches the warps' partials, so the
// cross-warp step costs one warp's work, not one per thread.  `buf`
// alternates the shared slots so that two barriers per reduction suffice.
struct RedShared {
    double2 part[2][32];
    double2 total[2];
};

template <typename VT>
__device__ __forceinline__ double2 block_sum2(DotAcc<VT> a, DotAcc<VT> b, RedShared &sh, int &buf)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    a.warp_reduce();
    b.warp_reduce();
    if (lane == 0) sh.part[buf][warp] = DotAcc<VT>::pack(a, b);
    __syncthreads();
    if (warp == 0) {
        DotAcc<VT> x, y;
        if (lane < nw) DotAcc<VT>::unpack(sh.part[buf][lane], x, y);
        x.warp_reduce();
        y.warp_reduce();
        if (lane == 0) sh.total[buf] = make_double2(x.value(), y.value());
    }
    __syncthreads();
    const double2 r = sh.total[buf];
    buf ^= 1;
    return r;
}
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

// ------------------------------------------------------------------ init
// k_1 = e_j / sqrt(S_jj); S k_1 = (column j of S) / sqrt(S_jj), read from block
// row j/4 (S is symmetric: S[4I+a][j] = S[j][4I+a]).
template <typename VT>
__global__ void init_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ Sv, const double *__restrict__ sdiag,
                            const int64_t *__restrict__ cols, VT *__restrict__ K,
                            VT *__restrict__ SK, int *__restrict__ status,
                            int *__restrict__ nu_eff, int nu, int64_t m_pad)
{
    const int c = blockIdx.x;
    const int64_t j = cols[c];
    const int64_t J = j >> 2;
    const int b = (int)(j & 3);
    VT *k0 = K + (int64_t)c * nu * m_pad;
    VT *sk0 = SK + (int64_t)c * nu * m_pad;
    for (int64_t r = threadIdx.x; r < m_pad; r += blockDim.x) {
        k0[r] = VT(0);
        sk0[r] = VT(0);
    }
    __syncthreads();
    const double inv = 1.0 / sqrt(sdiag[j]);
    if (threadIdx.x == 0) {
        k0[j] = (VT)inv;
        status[c] = 0;
        nu_eff[c] = nu;
    }
    for (int64_t k = rp[J] + threadIdx.x; k < rp[J + 1]; k += blockDim.x) {
        const int64_t I = ci[k];
#pragma unroll
        for (int a = 0; a < 4; ++a) sk0[4 * I + a] = (VT)(Sv[16 * k + 4 * b + a] * inv);
    }
}

// ------------------------------------------------------------------ SpMM
// Y[c] = A X[c] for the batch columns c < ncols.  Thread (tx, ty) of a 32x8 CTA
// owns block row I = 8 blockIdx.x + ty of column c = 32 blockIdx.y + tx, so
// the 32 lanes of a warp share block row I (the matrix block is a broadcast
// load) and read 32 columns' 4-vectors.  Rows run fastest in the grid, so the
// CTAs in flight work on one or two 32-column tiles whose input panels stay in
// L2 while their ~b gathers per entry hit it.
template <typename VT>
__global__ void __launch_bounds__(256) spmm_kernel(int64_t nbr, const int64_t *__restrict__ rp,
                                                   const int32_t *__restrict__ ci,
                                                   const VT *__restrict__ vals,
                                                   const VT *__restrict__ X, int64_t ldx,
                                                   VT *__restrict__ Y, int64_t ldy, int ncols)
{
    const int c = blockIdx.y * 32 + threadIdx.x;
    const int64_t I = (int64_t)blockIdx.x * 8 + threadIdx.y;
    if (c >= ncols || I >= nbr) return;
    const VT *x = X + (int64_t)c * ldx;
    VT acc[4] = {VT(0), VT(0), VT(0), VT(0)};
    const int64_t k1 = rp[I + 1];
    for (int64_t k = rp[I]; k < k1; ++k) {
        const VT *B = vals + 16 * k;
        VT r0[4], r1[4], r2[4], r3[4], xv[4];
        load4(B, r0);
        load4(B + 4, r1);
        load4(B + 8, r2);
        load4(B + 12, r3);
        load4(x + 4 * (int64_t)ci[k], xv);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            acc[0] = fma(r0[q], xv[q], acc[0]);
            acc[1] = fma(r1[q], xv[q], acc[1]);
            acc[2] = fma(r2[q], xv[q], acc[2]);
            acc[3] = fma(r3[q], xv[q], acc[3]);
        }
    }
    store4(Y + (int64_t)c * ldy + 4 * I, acc);
}

// ------------------------------------------------------------------ MGS
// One CTA per column; thread t owns entries r = t + v T (v < VPT) of the
// column's vectors.  Small VPT keeps w in registers.  VPT = 16 (m > 8192)
// keeps w in shared memory instead (1024 threads leave 64 registers each),
// with u in shared memory too when both fit, else re-read from global memory
// (an L2 hit: the SpMM has just written it).  Entries are visited in chunks
// with a compiler barrier between chunks so that only one chunk's loads are
// live per thread.  k_i is held across the reduction when it fits in
// registers, else re-read after it (an L2 hit).
template <typename VT, int VPT>
struct MgsCfg {
    static constexpr bool kWs = VPT >= 16;                                   // w in smem
    static constexpr bool kUs = !kWs || 2 * VPT * 1024 * sizeof(VT) <= 160 * 1024;  // u in smem
    static constexpr bool kHold = VPT * sizeof(VT) <= 64;
    static constexpr int kChunk = sizeof(VT) == 8 ? 4 : 8;
};

template <typename VT, int VPT>
__global__ void __launch_bounds__(1024, 1) mgs_kernel(const VT *__restrict__ K,
                                                      const VT *__restrict__ SK,
                                                      const VT *__restrict__ U,
                                                      VT *__restrict__ W,
                                                      double *__restrict__ Hsub,
                                                      double *__restrict__ cn2,
                                                      const int *__restrict__ status, int n,
                                                      int nu, int64_t m_pad, int need_w)
{
    using Cfg = MgsCfg<VT, VPT>;
    constexpr bool kWs = Cfg::kWs, kUs = Cfg::kUs, kHold = Cfg::kHold;
    constexpr int kChunk = Cfg::kChunk;
    const int c = blockIdx.x;
    if (status[c] != 0) return;
    // VPT >= 8 always runs 1024 threads: a compile-time T turns the per-entry
    // offsets v * T into load immediates instead of live registers.
    const int T = VPT >= 8 ? 1024 : (int)blockDim.x;
    const int tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT *us = reinterpret_cast<VT *>(smem_raw);             // u (if kUs)
    VT *ws = us + (kUs ? m_pad : 0);                        // w (if kWs)
    __shared__ RedShared red;
    __shared__ double ctot[kMaxNu];
    const int64_t base = (int64_t)c * nu * m_pad;
    const VT *u = U + (int64_t)c * m_pad;

    VT wr[kWs ? 1 : VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int r = tid + v * T;
        const VT x = u[r];
        if constexpr (kWs) ws[r] = x; else wr[v] = x;
        if constexpr (kUs) us[r] = x;
    }
    int buf = 0;
    // pass 1: h_{i,n} = k_i . u and the first Gram-Schmidt sweep
    for (int i = 0; i <= n; ++i) {
        const VT *ki = K + base + (int64_t)i * m_pad;
        const VT *ski = SK + base + (int64_t)i * m_pad;
        DotAcc<VT> ac, ah;
        VT kv[kHold ? VPT : 1];
#pragma unroll
        for (int v0 = 0; v0 < VPT; v0 += kChunk) {
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                const int v = v0 + q;
                if (v >= VPT) break;
                const int r = tid + v * T;
                const VT kr = ki[r];
                if constexpr (kHold) kv[v] = kr;
                VT uu;
                if constexpr (kUs) uu = us[r]; else uu = u[r];
                ah.add(kr, uu);
                if (need_w) {
                    VT wv;
                    if constexpr (kWs) wv = ws[r]; else wv = wr[v];
                    ac.add(ski[r], wv);
                }
            }
            if (v0 + kChunk < VPT) asm volatile("" ::: "memory");
        }
        const double2 s = block_sum2(ac, ah, red, buf);
        if (need_w) {
            const VT cc = (VT)s.x;
#pragma unroll
            for (int v0 = 0; v0 < VPT; v0 += kChunk) {
#pragma unroll
                for (int q = 0; q < kChunk; ++q) {
                    const int v = v0 + q;
                    if (v >= VPT) break;
                    const int r = tid + v * T;
                    VT kr;
                    if constexpr (kHold) kr = kv[v]; else kr = ki[r];
                    if constexpr (kWs) ws[r] = fma(-cc, kr, ws[r]); else wr[v] = fma(-cc, kr, wr[v]);
                }
                if (v0 + kChunk < VPT) asm volatile("" ::: "memory");
            }
        }
        if (tid == 0) {
            ctot[i] = s.x;
            Hsub[((int64_t)c * nu + i) * nu + n] = s.y;
            Hsub[((int64_t)c * nu + n) * nu + i] = s.y;
        }
    }
    if (!need_w) return;
    // pass 2: second Gram-Schmidt sweep
    for (int i = 0; i <= n; ++i) {
        const VT *ki = K + base + (int64_t)i * m_pad;
        const VT *ski = SK + base + (int64_t)i * m_pad;
        DotAcc<VT> ac;
        VT kv[kHold ? VPT : 1];
#pragma unroll
        for (int v0 = 0; v0 < VPT; v0 += kChunk) {
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                const int v = v0 + q;
                if (v >= VPT) break;
                const int r = tid + v * T;
                if constexpr (kHold) kv[v] = ki[r];
                VT wv;
                if constexpr (kWs) wv = ws[r]; else wv = wr[v];
                ac.add(ski[r], wv);
            }
            if (v0 + kChunk < VPT) asm volatile("" ::: "memory");
        }
        const double2 s = block_sum2(ac, DotAcc<VT>(), red, buf);
        const VT cc = (VT)s.x;
#pragma unroll
        for (int v0 = 0; v0 < VPT; v0 += kChunk) {
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                const int v = v0 + q;
                if (v >= VPT) break;
                const int r = tid + v * T;
                VT kr;
                if constexpr (kHold) kr = kv[v]; else kr = ki[r];
                if constexpr (kWs) ws[r] = fma(-cc, kr, ws[r]); else wr[v] = fma(-cc, kr, wr[v]);
            }
            if (v0 + kChunk < VPT) asm volatile("" ::: "memory");
        }
        if (tid == 0) ctot[i] += s.x;
    }
    VT *wo = W + (int64_t)c * m_pad;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int r = tid + v * T;
        if constexpr (kWs) wo[r] = ws[r]; else wo[r] = wr[v];
    }
    if (tid == 0) {
        double q = 0.0;
        for (int i = 0; i <= n; ++i) q += ctot[i] * ctot[i];
        cn2[c] = q;
    }
}

// ------------------------------------------------------------------ normalize
template <typename VT, int VPT>
__global__ void __launch_bounds__(1024) normalize_kernel(const VT *__restrict__ W,
                                                         const VT *__restrict__ SW,
                                                         VT *__restrict__ K, VT *__restrict__ SK,
                                                         const double *__restrict__ cn2,
                                                         int *__restrict__ status,
                                                         int *__restrict__ nu_eff, int n, int nu,
                                                         int64_t m_pad, double tau2)
{
    const int c = blockIdx.x;
    if (status[c] != 0) return;
    __shared__ RedShared red;
    const int T = VPT >= 8 ? 1024 : (int)blockDim.x, tid = threadIdx.x;
    const VT *w = W + (int64_t)c * m_pad;
    const VT *sw = SW + (int64_t)c * m_pad;
    DotAcc<VT> acc;
#pragma unroll 4
    for (int v = 0; v < VPT; ++v) acc.add(w[tid + v * T], sw[tid + v * T]);
    int buf = 0;
    const double beta2 = block_sum2(acc, DotAcc<VT>(), red, buf).x;
    VT *kn = K + ((int64_t)c * nu + n + 1) * m_pad;
    VT *skn = SK + ((int64_t)c * nu + n + 1) * m_pad;
    if (!(beta2 > 0.0) || beta2 <= tau2 * (beta2 + cn2[c])) {
        if (tid == 0) {
            status[c] = (beta2 >= 0.0) ? 1 : 2;   // 2: negative or NaN S-norm
            nu_eff[c] = n + 1;
        }
#pragma unroll 4
        for (int v = 0; v < VPT; ++v) {
            kn[tid + v * T] = VT(0);
            skn[tid + v * T] = VT(0);
        }
        return;
    }
    const double inv = 1.0 / sqrt(beta2);
    const VT vinv = (VT)inv;
#pragma unroll 4
    for (int v = 0; v < VPT; ++v) {
        if constexpr (sizeof(VT) == 8) {
            kn[tid + v * T] = w[tid + v * T] * vinv;
            skn[tid + v * T] = sw[tid + v * T] * vinv;
        } else {
            kn[tid + v * T] = (VT)((double)w[tid + v * T] * inv);
            skn[tid + v * T] = (VT)((double)sw[tid + v * T] * inv);
        }
    }
}

template <typename VT, int VPT>
cudaError_t mgs_dispatch(const KrylovBatch &b, int n, int need_w, cudaStream_t s)
{
    using Cfg = MgsCfg<VT, VPT>;
    const size_t smem = (size_t)b.shape.m_pad * sizeof(VT) * ((Cfg::kUs ? 1 : 0) + (Cfg::kWs ? 1 : 0));
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(mgs_kernel<VT, VPT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(kMaxGlobalM * sizeof(double)));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    mgs_kernel<VT, VPT><<<b.nb, b.shape.threads, smem, s>>>(
        (const VT *)b.K, (const VT *)b.SK, (const VT *)b.U, (VT *)b.W, b.Hsub, b.cn2, b.status, n,
        b.nu, b.shape.m_pad, need_w);
    return cudaGetLastError();
}

template <typename VT, int VPT>
cudaError_t normalize_dispatch(const KrylovBatch &b, int n, double tau, cudaStream_t s)
{
    normalize_kernel<VT, VPT><<<b.nb, b.shape.threads, 0, s>>>(
        (const VT *)b.W, (const VT *)b.SW, (VT *)b.K, (VT *)b.SK, b.cn2, b.status, b.nu_eff, n,
        b.nu, b.shape.m_pad, tau * tau);
    return cudaGetLastError();
}

template <typename VT>
cudaError_t mgs_vpt(const KrylovBatch &b, int n, int need_w, cudaStream_t s)
{
    switch (b.shape.vpt) {
    case 1: return mgs_dispatch<VT, 1>(b, n, need_w, s);
    case 2: return mgs_dispatch<VT, 2>(b, n, need_w, s);
    case 4: return mgs_dispatch<VT, 4>(b, n, need_w, s);
    case 8: return mgs_dispatch<VT, 8>(b, n, need_w, s);
    case 16: return mgs_dispatch<VT, 16>(b, n, need_w, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename VT>
cudaError_t normalize_vpt(const KrylovBatch &b, int n, double tau, cudaStream_t s)
{
    switch (b.shape.vpt) {
    case 1: return normalize_dispatch<VT, 1>(b, n, tau, s);
    case 2: return normalize_dispatch<VT, 2>(b, n, tau, s);
    case 4: return normalize_dispatch<VT, 4>(b, n, tau, s);
    case 8: return normalize_dispatch<VT, 8>(b, n, tau, s);
    case 16: return normalize_dispatch<VT, 16>(b, n, tau, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_init(const DeviceMatrix &A, const KrylovBatch &b, cudaStream_t s)
{
    if (b.prec == 0)
        init_kernel<double><<<b.nb, 256, 0, s>>>(A.rp, A.ci, A.Sd, A.sdiag, b.cols, (double *)b.K,
                                                 (double *)b.SK, b.status, b.nu_eff, b.nu,
                                                 b.shape.m_pad);
    else
        init_kernel<float><<<b.nb, 256, 0, s>>>(A.rp, A.ci, A.Sd, A.sdiag, b.cols, (float *)b.K,
                                                (float *)b.SK, b.status, b.nu_eff, b.nu,
                                                b.shape.m_pad);
    return cudaGetLastError();
}

cudaError_t launch_spmm(const DeviceMatrix &A, int which, const KrylovBatch &b, const void *X,
                        int64_t ldx, void *Y, int64_t ldy, cudaStream_t s)
{
    const dim3 block(32, 8);
    const dim3 grid((unsigned)((A.nbr + 7) / 8), (unsigned)((b.nb + 31) / 32));
    if (b.prec == 0)
        spmm_kernel<double><<<grid, block, 0, s>>>(A.nbr, A.rp, A.ci, which ? A.Sd : A.Hd,
                                                   (const double *)X, ldx, (double *)Y, ldy, b.nb);
    else
        spmm_kernel<float><<<grid, block, 0, s>>>(A.nbr, A.rp, A.ci, which ? A.Sf : A.Hf,
                                                  (const float *)X, ldx, (float *)Y, ldy, b.nb);
    return cudaGetLastError();
}

cudaError_t launch_mgs(const KrylovBatch &b, int n, int need_w, cudaStream_t s)
{
    return b.prec == 0 ? mgs_vpt<double>(b, n, need_w, s) : mgs_vpt<float>(b, n, need_w, s);
}

cudaError_t launch_normalize(const KrylovBatch &b, int n, double tau, cudaStream_t s)
{
    return b.prec == 0 ? normalize_vpt<double>(b, n, tau, s) : normalize_vpt<float>(b, n, tau, s);
}

}  // namespace marnoldi
