// Krylov-subspace build of the multiple Arnoldi method on sm_103a.
//
// For a batch of columns j, builds the S-orthonormal basis K of
// span{e_j, H e_j, ..., H^(nu-1) e_j} (arXiv:1307.3218, Section 2: the subspace
// L_nu^(j) containing e_j whose nu x nu *standard* eigenproblem replaces
// H phi = eps S phi, Eq. 2) and the explicit subspace matrix H_sub = K^T H K.
//
// The basis is stored unnormalised: slot i holds w_i and S w_i, and
// k_i = s_i w_i with s_i = 1 / ||w_i||_S.  One Krylov step n, for every column:
//   spmm(H):    H w_n                                    (BSR 4x4 x batch panel)
//   mgs:        beta_n = sqrt(w_n . S w_n); stop the column when
//               beta_n^2 <= tau^2 (beta_n^2 + sum_i c_i^2), i.e.
//               ||w_n||_S <= tau ||u_{n-1}||_S (S-orthogonality of K splits
//               ||u||_S^2 into beta^2 plus the squared projection coefficients);
//               else s_n = 1 / beta_n, u = s_n H w_n, h_{i,n} = k_i . u (i <= n),
//               and two passes of modified Gram-Schmidt in the S inner product
//               using the stored S w_i: c_i = (S k_i) . w, w -= c_i k_i;
//               w is written to slot n+1
//   spmm(S):    S w into slot n+1
//
// Inner products are always accumulated to FP64 accuracy; in mixed precision
// the vectors, the SpMM and the Gram-Schmidt updates are FP32.  Reductions use
// a fixed order (warp butterfly, then warp 0 over the warps), so results do not
// depend on scheduling.
#include "internal.h"

#include <cstdio>

namespace marnoldi {

const char *kernel_name(int kind)
{
    static const char *names[KK_NKINDS] = {"init",   "spmm_H", "mgs",     "spmm_S", "eigsub",
                                           "minmax", "count",  "density", "green", "region"};
    return (kind >= 0 && kind < KK_NKINDS) ? names[kind] : "?";
}

// Vectors up to 4096 entries run 256-thread CTAs (several columns share an SM
// and overlap each other's barriers); longer ones 1024-thread CTAs.  VPT is
// the power of two that covers m.
ColumnShape column_shape(int64_t m)
{
    const int T = m <= 4096 ? 256 : 1024;
    int v = 1;
    while (v < 16 && (int64_t)v * T < m) v *= 2;
    return ColumnShape{v, T, (int64_t)v * T};
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
// butterflies, then warp 0 over the warps' partials).  Thread 0 of warp 0 runs
// `epi(totals, slot)` before the final barrier: the scalar FP64 work that
// follows a reduction (scales, coefficients, the breakdown test) is done once
// there and handed to the CTA through shared memory, instead of by every
// thread on GB300's narrow FP64 pipe.  `buf` alternates the shared slots so
// that two barriers per reduction suffice.
struct RedShared {
    double2 part[2][32];
    double2 total[2];
};

struct NoEpilogue {
    __device__ __forceinline__ void operator()(double2, int) const {}
};

template <typename VT, typename Epi = NoEpilogue>
__device__ __forceinline__ double2 block_sum2(DotAcc<VT> a, DotAcc<VT> b, RedShared &sh, int &buf,
                                              Epi epi = Epi())
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
        if (lane == 0) {
            const double2 t = make_double2(x.value(), y.value());
            sh.total[buf] = t;
            epi(t, buf);
        }
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
                            VT *__restrict__ SK, double *__restrict__ scale,
                            int *__restrict__ status, int *__restrict__ nu_eff, int nu,
                            int64_t m_pad)
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
        scale[(int64_t)c * nu] = 1.0;
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

// Mixed precision, matrix blocks stored as 16 "hi" then 16 "lo" FP32 values
// (hi + lo = the FP64 value to about 2^-48; one 128-byte line per block).
//
// S w (spmm_f32_kernel): plain FP32 with the hi values.  Its rounding only
// perturbs the Gram-Schmidt coefficients and the norms, which the second pass
// and the subspace Galerkin step absorb.
//
// H w (spmm_f32_accurate_kernel): the subspace matrix entries h_{i,n} = k_i . u
// take u = H k_n at face value, so u is formed to about 2^-48: each product
// with hi is split exactly (p + e, e = fma(h, x, -p)) and summed with exact
// two-sums, the lo products and the errors collect in a second FP32 word, and
// u is written as a normalised (hi, lo) FP32 pair.  The Krylov vector itself
// continues from the hi word.  The extra FP32 work is hidden behind the
// gather, which bounds this kernel.
__global__ void __launch_bounds__(256) spmm_f32_kernel(int64_t nbr, const int64_t *__restrict__ rp,
                                                       const int32_t *__restrict__ ci,
                                                       const float *__restrict__ vals,
                                                       const float *__restrict__ X, int64_t ldx,
                                                       float *__restrict__ Y, int64_t ldy, int ncols)
{
    const int c = blockIdx.y * 32 + threadIdx.x;
    const int64_t I = (int64_t)blockIdx.x * 8 + threadIdx.y;
    if (c >= ncols || I >= nbr) return;
    const float *x = X + (int64_t)c * ldx;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int64_t k1 = rp[I + 1];
    for (int64_t k = rp[I]; k < k1; ++k) {
        const float *B = vals + 32 * k;
        float r0[4], r1[4], r2[4], r3[4], xv[4];
        load4(x + 4 * (int64_t)ci[k], xv);
        load4(B, r0);
        load4(B + 4, r1);
        load4(B + 8, r2);
        load4(B + 12, r3);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            acc[0] = fmaf(r0[q], xv[q], acc[0]);
            acc[1] = fmaf(r1[q], xv[q], acc[1]);
            acc[2] = fmaf(r2[q], xv[q], acc[2]);
            acc[3] = fmaf(r3[q], xv[q], acc[3]);
        }
    }
    store4(Y + (int64_t)c * ldy + 4 * I, acc);
}

__global__ void __launch_bounds__(256) spmm_f32_accurate_kernel(
    int64_t nbr, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
    const float *__restrict__ vals, const float *__restrict__ X, int64_t ldx,
    float *__restrict__ Y, float *__restrict__ Ylo, int64_t ldy, int ncols)
{
    const int c = blockIdx.y * 32 + threadIdx.x;
    const int64_t I = (int64_t)blockIdx.x * 8 + threadIdx.y;
    if (c >= ncols || I >= nbr) return;
    const float *x = X + (int64_t)c * ldx;
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    const int64_t k1 = rp[I + 1];
    for (int64_t k = rp[I]; k < k1; ++k) {
        const float *B = vals + 32 * k;
        float xv[4];
        load4(x + 4 * (int64_t)ci[k], xv);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            float h[4], l[4];
            load4(B + 4 * a, h);
            load4(B + 16 + 4 * a, l);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float p = __fmul_rn(h[q], xv[q]);
                const float e = __fmaf_rn(h[q], xv[q], -p);
                df_add(hi[a], lo[a], p, __fmaf_rn(l[q], xv[q], e));
            }
        }
    }
    float yh[4], yl[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {   // renormalise: yh = fl(hi + lo), yl = the rest
        yh[a] = __fadd_rn(hi[a], lo[a]);
        yl[a] = __fsub_rn(lo[a], __fsub_rn(yh[a], hi[a]));
    }
    store4(Y + (int64_t)c * ldy + 4 * I, yh);
    store4(Ylo + (int64_t)c * ldy + 4 * I, yl);
}

// Mixed precision over row tiles.  Rows adjacent in the (spatially sorted)
// atom order share most of their neighbours, so a CTA stages the x entries of
// its tile's neighbour union for its 32 columns in shared memory once (each
// 16-byte entry gathered once instead of once per block that uses it: about
// 3x fewer gathers on amorphous carbon), then every warp computes its rows
// from shared memory.  Lanes are columns, as above, so the staged entries are
// read without bank conflicts and the matrix block stays a broadcast load.
// MODE 0: plain FP32 with the hi values (S); MODE 1: exact products and
// two-sums over hi + lo with a (hi, lo) output (H).
template <int MODE>
__global__ void __launch_bounds__(256) spmm_tile_kernel(
    const int *__restrict__ tile_row0, const int *__restrict__ tile_uptr,
    const int *__restrict__ tile_u, const uint8_t *__restrict__ blk_u,
    const int64_t *__restrict__ rp, const float *__restrict__ vals, const float *__restrict__ X,
    int64_t ldx, float *__restrict__ Y, float *__restrict__ Ylo, int64_t ldy, int ncols)
{
    extern __shared__ __align__(16) float4 xs[];   // [kTileCap][32]
    const int tile = blockIdx.x, lane = threadIdx.x, warp = threadIdx.y;
    const int c = blockIdx.y * 32 + lane;
    const bool live = c < ncols;
    const int u0 = tile_uptr[tile], nt = tile_uptr[tile + 1] - u0;
    const float *x = X + (int64_t)(live ? c : 0) * ldx;
    for (int u = warp; u < nt; u += 8) {
        const int J = tile_u[u0 + u];
        xs[u * 32 + lane] = live ? __ldg(reinterpret_cast<const float4 *>(x + 4 * (int64_t)J))
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const int I1 = tile_row0[tile + 1];
    for (int I = tile_row0[tile] + warp; I < I1; I += 8) {
        float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
        const int64_t k1 = rp[I + 1];
        for (int64_t k = rp[I]; k < k1; ++k) {
            const float4 x4 = xs[(int)blk_u[k] * 32 + lane];
            const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
            const float *B = vals + 32 * k;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                float h[4];
                load4(B + 4 * a, h);
                if constexpr (MODE == 1) {
                    float l[4];
                    load4(B + 16 + 4 * a, l);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float p = __fmul_rn(h[q], xv[q]);
                        const float e = __fmaf_rn(h[q], xv[q], -p);
                        df_add(hi[a], lo[a], p, __fmaf_rn(l[q], xv[q], e));
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) hi[a] = fmaf(h[q], xv[q], hi[a]);
                }
            }
        }
        if (!live) continue;
        if constexpr (MODE == 1) {
            float yh[4], yl[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                yh[a] = __fadd_rn(hi[a], lo[a]);
                yl[a] = __fsub_rn(lo[a], __fsub_rn(yh[a], hi[a]));
            }
            store4(Y + (int64_t)c * ldy + 4 * I, yh);
            store4(Ylo + (int64_t)c * ldy + 4 * I, yl);
        } else {
            store4(Y + (int64_t)c * ldy + 4 * I, hi);
        }
    }
}

// ------------------------------------------------------------------ MGS
// One CTA of T threads per column; thread t owns entries r = t + v T
// (v < VPT) of the column's vectors.  T is a compile-time constant, so the
// per-entry offsets v T are load immediates rather than live registers.
// Small VPT keeps w in registers; VPT = 16 keeps w in shared memory instead
// (64 registers per thread do not hold it), with u in shared memory too when
// both fit, else re-read from global memory (an L2 hit: the SpMM has just
// written it).  Entries are visited in chunks with a compiler barrier between
// chunks so that only one chunk's loads are live per thread.  The stored w_i
// is held across the reduction when it fits in registers, else re-read after
// it (an L2 hit).
template <typename VT, int VPT, int T>
struct MgsCfg {
    static constexpr bool kLo = sizeof(VT) == 4;                    // u as (hi, lo) pair
    static constexpr bool kWs = VPT >= 16;                          // w in smem
    static constexpr bool kUs = kLo || !kWs || 2 * VPT * T * sizeof(VT) <= 160 * 1024;
    static constexpr bool kHold = VPT * sizeof(VT) <= 64;
    static constexpr int kChunk = sizeof(VT) == 8 ? 4 : 8;
    static constexpr int kSmemVectors = (kUs ? 1 : 0) + (kLo ? 1 : 0) + (kWs ? 1 : 0);
};

// w -= a x over the thread's entries (x from registers or re-read).
template <typename VT, int VPT, int kChunk, bool kHold, bool kWs>
__device__ __forceinline__ void axpy_entries(VT (&wr)[kWs ? 1 : VPT], VT *ws,
                                             const VT (&kv)[kHold ? VPT : 1],
                                             const VT *__restrict__ x, int tid, int T, VT a)
{
#pragma unroll
    for (int v0 = 0; v0 < VPT; v0 += kChunk) {
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int v = v0 + q;
            if (v >= VPT) break;
            const int r = tid + v * T;
            VT kr;
            if constexpr (kHold) kr = kv[v]; else kr = x[r];
            if constexpr (kWs) ws[r] = fma(-a, kr, ws[r]); else wr[v] = fma(-a, kr, wr[v]);
        }
        if (v0 + kChunk < VPT) asm volatile("" ::: "memory");
    }
}

template <typename VT, int VPT, int T>
__global__ void __launch_bounds__(T, T == 256 ? 4 : 1) mgs_kernel(
    VT *__restrict__ K, VT *__restrict__ SK, const VT *__restrict__ U, const VT *__restrict__ Ulo,
    double *__restrict__ Hsub, double *__restrict__ scale, double *__restrict__ cn2,
    int *__restrict__ status, int *__restrict__ nu_eff, int n, int nu, int64_t m_pad, int need_w,
    double tau2)
{
    using Cfg = MgsCfg<VT, VPT, T>;
    constexpr bool kWs = Cfg::kWs, kUs = Cfg::kUs, kHold = Cfg::kHold, kLo = Cfg::kLo;
    constexpr int kChunk = Cfg::kChunk;
    const int c = blockIdx.x;
    if (status[c] != 0) return;
    const int tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT *us = reinterpret_cast<VT *>(smem_raw);             // u = H w_n, unscaled (if kUs)
    VT *uls = us + (kUs ? m_pad : 0);                       // its lo word (mixed precision)
    VT *ws = uls + (kLo ? m_pad : 0);                       // w (if kWs)
    __shared__ RedShared red;
    __shared__ double ctot[kMaxNu];
    __shared__ double ssc[kMaxNu];
    __shared__ VT bc_coef[2];     // the FP32/FP64 update coefficient of the last reduction
    __shared__ double bc_sn;
    __shared__ int bc_stop;
    const int64_t base = (int64_t)c * nu * m_pad;
    int buf = 0;

    for (int i = tid; i < n; i += T) ssc[i] = scale[(int64_t)c * nu + i];
    // beta_n = ||w_n||_S and the breakdown test (slot 0 is stored normalised)
    double sn = 1.0;
    if (n > 0) {
        const VT *wn = K + base + (int64_t)n * m_pad;
        const VT *swn = SK + base + (int64_t)n * m_pad;
        DotAcc<VT> acc;
#pragma unroll
        for (int v0 = 0; v0 < VPT; v0 += kChunk) {
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                const int v = v0 + q;
                if (v >= VPT) break;
                acc.add(wn[tid + v * T], swn[tid + v * T]);
            }
            if (v0 + kChunk < VPT) asm volatile("" ::: "memory");
        }
        block_sum2(acc, DotAcc<VT>(), red, buf, [&](double2 t, int) {
            const double beta2 = t.x;
            if (!(beta2 > 0.0) || beta2 <= tau2 * (beta2 + cn2[c])) {
                status[c] = (beta2 >= 0.0) ? 1 : 2;   // 2: negative or NaN S-norm
                nu_eff[c] = n;
                bc_stop = 1;
            } else {
                const double s = 1.0 / sqrt(beta2);
                scale[(int64_t)c * nu + n] = s;
                bc_sn = s;
                bc_stop = 0;
            }
        });
        if (bc_stop) return;   // uniform: read after the reduction's last barrier
        sn = bc_sn;
    }
    __syncthreads();   // ssc visible
    // w starts as u = s_n H w_n; the h dots use H w_n unscaled (with its lo
    // word in mixed precision) and apply s_i s_n in FP64 after the reduction
    const VT vsn = (VT)sn;
    const VT *u = U + (int64_t)c * m_pad;
    const VT *ul = kLo ? Ulo + (int64_t)c * m_pad : nullptr;
    VT wr[kWs ? 1 : VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int r = tid + v * T;
        const VT x = u[r];
        if constexpr (kWs) ws[r] = x * vsn; else wr[v] = x * vsn;
        if constexpr (kUs) us[r] = x;
        if constexpr (kLo) uls[r] = ul[r];
    }
    // pass 1: h_{i,n} = k_i . u and the first Gram-Schmidt sweep
    for (int i = 0; i <= n; ++i) {
        const double si = i == n ? sn : ssc[i];
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
                if constexpr (kLo) ah.add(kr, uls[r]);
                if (need_w) {
                    VT wv;
                    if constexpr (kWs) wv = ws[r]; else wv = wr[v];
                    ac.add(ski[r], wv);
                }
            }
            if (v0 + kChunk < VPT) asm volatile("" ::: "memory");
        }
        block_sum2(ac, ah, red, buf, [&](double2 t, int slot) {
            const double ci = t.x * si, h = t.y * si * sn;
            ctot[i] = ci;
            bc_coef[slot] = (VT)(ci * si);
            Hsub[((int64_t)c * nu + i) * nu + n] = h;
            Hsub[((int64_t)c * nu + n) * nu + i] = h;
        });
        if (need_w)
            axpy_entries<VT, VPT, kChunk, kHold, kWs>(wr, ws, kv, ki, tid, T, bc_coef[buf ^ 1]);
    }
    if (!need_w) return;
    // pass 2: second Gram-Schmidt sweep
    for (int i = 0; i <= n; ++i) {
        const double si = i == n ? sn : ssc[i];
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
        block_sum2(ac, DotAcc<VT>(), red, buf, [&](double2 t, int slot) {
            const double ci = t.x * si;
            ctot[i] += ci;
            bc_coef[slot] = (VT)(ci * si);
        });
        axpy_entries<VT, VPT, kChunk, kHold, kWs>(wr, ws, kv, ki, tid, T, bc_coef[buf ^ 1]);
    }
    VT *wo = K + base + (int64_t)(n + 1) * m_pad;   // the next slot, unnormalised
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

template <typename VT, int VPT, int T>
cudaError_t mgs_dispatch(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s)
{
    using Cfg = MgsCfg<VT, VPT, T>;
    const size_t smem = (size_t)b.shape.m_pad * sizeof(VT) * Cfg::kSmemVectors;
    static bool configured = false;
    if (!configured) {
        const int maxs = (int)((size_t)VPT * T * sizeof(VT) * Cfg::kSmemVectors);
        cudaError_t e = cudaFuncSetAttribute(mgs_kernel<VT, VPT, T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    mgs_kernel<VT, VPT, T><<<b.nb, T, smem, s>>>(
        (VT *)b.K, (VT *)b.SK, (const VT *)b.U, (const VT *)b.Ulo, b.Hsub, b.scale, b.cn2,
        b.status, b.nu_eff, n, b.nu, b.shape.m_pad, need_w, tau * tau);
    return cudaGetLastError();
}

template <typename VT>
cudaError_t mgs_shape(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s)
{
    if (b.shape.threads == 1024) {
        switch (b.shape.vpt) {
        case 1: return mgs_dispatch<VT, 1, 1024>(b, n, need_w, tau, s);
        case 2: return mgs_dispatch<VT, 2, 1024>(b, n, need_w, tau, s);
        case 4: return mgs_dispatch<VT, 4, 1024>(b, n, need_w, tau, s);
        case 8: return mgs_dispatch<VT, 8, 1024>(b, n, need_w, tau, s);
        case 16: return mgs_dispatch<VT, 16, 1024>(b, n, need_w, tau, s);
        default: return cudaErrorInvalidValue;
        }
    }
    if (b.shape.threads != 256) return cudaErrorInvalidValue;
    switch (b.shape.vpt) {
    case 1: return mgs_dispatch<VT, 1, 256>(b, n, need_w, tau, s);
    case 2: return mgs_dispatch<VT, 2, 256>(b, n, need_w, tau, s);
    case 4: return mgs_dispatch<VT, 4, 256>(b, n, need_w, tau, s);
    case 8: return mgs_dispatch<VT, 8, 256>(b, n, need_w, tau, s);
    case 16: return mgs_dispatch<VT, 16, 256>(b, n, need_w, tau, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_init(const DeviceMatrix &A, const KrylovBatch &b, cudaStream_t s)
{
    if (b.prec == 0)
        init_kernel<double><<<b.nb, 256, 0, s>>>(A.rp, A.ci, A.Sd, A.sdiag, b.cols, (double *)b.K,
                                                 (double *)b.SK, b.scale, b.status, b.nu_eff, b.nu,
                                                 b.shape.m_pad);
    else
        init_kernel<float><<<b.nb, 256, 0, s>>>(A.rp, A.ci, A.Sd, A.sdiag, b.cols, (float *)b.K,
                                                (float *)b.SK, b.scale, b.status, b.nu_eff, b.nu,
                                                b.shape.m_pad);
    return cudaGetLastError();
}

cudaError_t launch_spmm(const DeviceMatrix &A, int which, const KrylovBatch &b, const void *X,
                        int64_t ldx, void *Y, int64_t ldy, cudaStream_t s)
{
    const dim3 block(32, 8);
    // The staged tile form pays off for the gather-bound plain S product; the
    // accurate H product is bound by its exact-arithmetic FP32 work and runs
    // faster in the direct form below.
    if (b.prec == 1 && A.ntiles > 0 && which == 1) {
        const size_t smem = (size_t)kTileCap * 32 * sizeof(float4);
        static bool configured = false;
        if (!configured) {
            cudaError_t e = cudaFuncSetAttribute(spmm_tile_kernel<0>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(spmm_tile_kernel<1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            configured = true;
        }
        const dim3 tgrid((unsigned)A.ntiles, (unsigned)((b.nb + 31) / 32));
        if (which == 0)
            spmm_tile_kernel<1><<<tgrid, block, smem, s>>>(A.tile_row0, A.tile_uptr, A.tile_u, A.blk_u,
                                                           A.rp, A.Hf, (const float *)X, ldx, (float *)Y,
                                                           (float *)b.Ulo, ldy, b.nb);
        else
            spmm_tile_kernel<0><<<tgrid, block, smem, s>>>(A.tile_row0, A.tile_uptr, A.tile_u, A.blk_u,
                                                           A.rp, A.Sf, (const float *)X, ldx, (float *)Y,
                                                           nullptr, ldy, b.nb);
        return cudaGetLastError();
    }
    const dim3 grid((unsigned)((A.nbr + 7) / 8), (unsigned)((b.nb + 31) / 32));
    if (b.prec == 0)
        spmm_kernel<double><<<grid, block, 0, s>>>(A.nbr, A.rp, A.ci, which ? A.Sd : A.Hd,
                                                   (const double *)X, ldx, (double *)Y, ldy, b.nb);
    else if (which == 0)
        spmm_f32_accurate_kernel<<<grid, block, 0, s>>>(A.nbr, A.rp, A.ci, A.Hf, (const float *)X,
                                                        ldx, (float *)Y, (float *)b.Ulo, ldy, b.nb);
    else
        spmm_f32_kernel<<<grid, block, 0, s>>>(A.nbr, A.rp, A.ci, A.Sf, (const float *)X, ldx,
                                               (float *)Y, ldy, b.nb);
    return cudaGetLastError();
}

cudaError_t launch_mgs(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s)
{
    return b.prec == 0 ? mgs_shape<double>(b, n, need_w, tau, s) : mgs_shape<float>(b, n, need_w, tau, s);
}

}  // namespace marnoldi
