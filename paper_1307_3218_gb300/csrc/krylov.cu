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
                                           "minmax", "count",  "density", "green", "region", "support", "spmm_HS"};
    return (kind >= 0 && kind < KK_NKINDS) ? names[kind] : "?";
}

// Vectors up to 4096 entries run 256-thread CTAs (several columns share an SM
// and overlap each other's reductions).  Longer FP32 vectors up to 8192
// entries run 512-thread CTAs of 16 values per thread (two per SM); the rest
// run 1024-thread CTAs.  VPT is the power of two that covers m.
ColumnShape column_shape(int64_t m, int prec)
{
    if (prec == 1 && m > 4096 && m <= 8192) return ColumnShape{16, 512, 8192};
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
    __device__ __forceinline__ void merge(const DotAcc &o) { s += o.s; }
    __device__ __forceinline__ DotAcc shfl_xor(int o) const
    {
        DotAcc r;
        r.s = __shfl_xor_sync(kFull, s, o);
        return r;
    }
    __device__ __forceinline__ double pack() const { return s; }
    __device__ __forceinline__ void unpack(double p) { s = p; }
    __device__ __forceinline__ void set(double x) { s = x; }
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
    // fold in a correction of about 2^-24 relative to the sum
    __device__ __forceinline__ void add_lo(float x) { lo = __fadd_rn(lo, x); }
    __device__ __forceinline__ void merge(const DotAcc &o) { df_add(hi, lo, o.hi, o.lo); }
    __device__ __forceinline__ DotAcc shfl_xor(int o) const
    {
        DotAcc r;
        r.hi = __shfl_xor_sync(kFull, hi, o);
        r.lo = __shfl_xor_sync(kFull, lo, o);
        return r;
    }
    __device__ __forceinline__ double pack() const
    {
        union { float2 f; double d; } u;
        u.f = make_float2(hi, lo);
        return u.d;
    }
    __device__ __forceinline__ void unpack(double p)
    {
        union { float2 f; double d; } u;
        u.d = p;
        hi = u.f.x;
        lo = u.f.y;
    }
    __device__ __forceinline__ void set(float x)
    {
        hi = x;
        lo = 0.f;
    }
};

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
// Entries are stored at their positions in the column's tile order.
template <typename VT>
__global__ void init_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ Sv, const double *__restrict__ sdiag,
                            const int64_t *__restrict__ cols, VT *__restrict__ K,
                            VT *__restrict__ SK, double *__restrict__ scale,
                            int *__restrict__ status, int *__restrict__ nu_eff, int nu,
                            int64_t m_pad, const uint16_t *__restrict__ tinv, int nb)
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
        k0[vpos(tinv, nb, c, j)] = (VT)inv;
        scale[(int64_t)c * nu] = 1.0;
        status[c] = 0;
        nu_eff[c] = nu;
    }
    for (int64_t k = rp[J] + threadIdx.x; k < rp[J + 1]; k += blockDim.x) {
        const int64_t I = ci[k];
#pragma unroll
        for (int a = 0; a < 4; ++a) sk0[vpos(tinv, nb, c, 4 * I + a)] = (VT)(Sv[16 * k + 4 * b + a] * inv);
    }
}

// ------------------------------------------------------------------ SpMM
// Y[c] = A X[c] for the batch columns c < ncols.  Thread (tx, ty) of a 32x8 CTA
// owns block row I = 8 blockIdx.x + ty of column c = 32 blockIdx.y + tx, so
// the 32 lanes of a warp share block row I (the matrix block is a broadcast
// load) and read 32 columns' 4-vectors, and the CTA's 8 rows are support tile
// blockIdx.x.  Rows run fastest in the grid, so the CTAs in flight work on one
// or two 32-column tiles whose input panels stay in L2 while their ~b gathers
// per entry hit it.
//
// Column c's x and y are stored in its tile order: block row I at position
// apos(I) = 8 tinv[I / 8] + I % 8 (4 entries each).  Support: row I of
// column c vanishes when its tile lies more than `lim` hops from the column's
// atom (thop > lim; the input vanishes beyond lim - 1).  A lane past the
// support gathers nothing and a warp with no live lane only writes its zeros.
struct RowLive {
    bool live, act;
};
__device__ __forceinline__ RowLive row_live(const uint8_t *__restrict__ thop, int tile, int nb,
                                            int c, int lim)
{
    const bool live = c < nb;
    return RowLive{live, live && (int)thop[(int64_t)tile * nb + c] <= lim};
}
__device__ __forceinline__ int64_t apos(const uint16_t *__restrict__ tinv, int nb, int c, int64_t I)
{
    return 8 * (int64_t)tinv[(I >> 3) * nb + c] + (I & 7);
}

// H x and S x for the same panel in one pass (both feed the Gram-Schmidt step
// of the same Krylov vector, and H and S share their block pattern): each x
// entry is gathered once for both products.  Thread (tx, ty) of a 32x8 CTA
// owns block row I = 8 blockIdx.x + ty (the CTA's 8 rows are support tile
// blockIdx.x) for the two columns c = 64 blockIdx.y + tx and c + 32, so every
// matrix block, a broadcast load across the warp, serves 64 columns.  Rows run
// fastest in the grid, so the CTAs in flight work on one or two 64-column
// tiles whose input panels stay in L2 while their ~b gathers per entry hit it.
//
// FP64: plain FMAs.  Mixed precision (matrix blocks stored as 16 "hi" then 16
// "lo" FP32 values, hi + lo = the FP64 value to about 2^-48): the subspace
// matrix entries h_{i,n} = k_i . u take u = H k_n at face value, so u is
// formed to about 2^-48: each product with hi is split exactly (p + e,
// e = fma(h, x, -p)) and summed with exact two-sums, the lo products and the
// errors collect in a second FP32 word, and u is written as a normalised
// (hi, lo) FP32 pair; the Krylov vector itself continues from the hi word.
// S x is plain FP32 with the hi values: its rounding only perturbs the
// Gram-Schmidt coefficients and the norms, which the second pass and the
// subspace Galerkin step absorb.
template <typename VT, bool kS>
__global__ void __launch_bounds__(256) spmm_hs_kernel(
    int64_t nbr, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
    const VT *__restrict__ Hv, const VT *__restrict__ Sv, const VT *__restrict__ X, int64_t ldx,
    VT *__restrict__ U, VT *__restrict__ Ulo, int64_t ldu, VT *__restrict__ SY, int64_t ldsy,
    int ncols, const uint8_t *__restrict__ thop, const uint16_t *__restrict__ tinv, int lim)
{
    constexpr bool kF = sizeof(VT) == 4;
    constexpr int BS = kF ? 32 : 16;   // stored values per block
    const int64_t I = (int64_t)blockIdx.x * 8 + threadIdx.y;
    if (I >= nbr) return;   // uniform over the warp
    int cc[2];
    RowLive L[2];
    int64_t yo[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        cc[h] = blockIdx.y * 64 + 32 * h + threadIdx.x;
        L[h] = row_live(thop, blockIdx.x, ncols, cc[h], lim);
        yo[h] = L[h].live ? 4 * apos(tinv, ncols, cc[h], I) : 0;
    }
    VT hi[2][4], lo[2][4], sy[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int a = 0; a < 4; ++a) hi[h][a] = lo[h][a] = sy[h][a] = VT(0);
    if (__any_sync(kFull, L[0].act || L[1].act)) {
        const VT *x0 = X + (int64_t)(L[0].live ? cc[0] : 0) * ldx;
        const VT *x1 = X + (int64_t)(L[1].live ? cc[1] : 0) * ldx;
        const int64_t k1 = rp[I + 1];
        for (int64_t k = rp[I]; k < k1; ++k) {
            const int64_t J = ci[k];
            VT xv[2][4] = {{VT(0), VT(0), VT(0), VT(0)}, {VT(0), VT(0), VT(0), VT(0)}};
            if (L[0].act) load4(x0 + 4 * apos(tinv, ncols, cc[0], J), xv[0]);
            if (L[1].act) load4(x1 + 4 * apos(tinv, ncols, cc[1], J), xv[1]);
            const VT *Hb = Hv + BS * k;
            const VT *Sb = Sv + BS * k;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                VT hr[4], sr[4], lr[4];
                load4(Hb + 4 * a, hr);
                if constexpr (kS) load4(Sb + 4 * a, sr);
                if constexpr (kF) load4(Hb + 16 + 4 * a, lr);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if constexpr (kF) {
                            const float p = __fmul_rn(hr[q], xv[h][q]);
                            const float e = __fmaf_rn(hr[q], xv[h][q], -p);
                            df_add(hi[h][a], lo[h][a], p, __fmaf_rn(lr[q], xv[h][q], e));
                        } else {
                            hi[h][a] = fma(hr[q], xv[h][q], hi[h][a]);
                        }
                        if constexpr (kS) sy[h][a] = fma(sr[q], xv[h][q], sy[h][a]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!L[h].live) continue;
        if constexpr (kF) {
            float yh[4], yl[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {   // renormalise: yh = fl(hi + lo), yl = the rest
                yh[a] = __fadd_rn(hi[h][a], lo[h][a]);
                yl[a] = __fsub_rn(lo[h][a], __fsub_rn(yh[a], hi[h][a]));
            }
            store4(U + (int64_t)cc[h] * ldu + yo[h], yh);
            store4(Ulo + (int64_t)cc[h] * ldu + yo[h], yl);
        } else {
            store4(U + (int64_t)cc[h] * ldu + yo[h], hi[h]);
        }
        if constexpr (kS) store4(SY + (int64_t)cc[h] * ldsy + yo[h], sy[h]);
    }
}

// ------------------------------------------------------------------ MGS
// One CTA of T threads (NW = T / 32 warps) per column; thread t owns the
// values at positions p = t + v T (v < VPT) of the column's vectors, which are
// stored in the column's tile order (tiles of 32 entries by hop count from the
// column's atom).  Position tile k = w + NW v belongs to warp w, and vector i
// vanishes past the first tcnt[i + 1] tiles (S w_i reaches one hop further
// than w_i), so a warp's live values for vector i are its first
// nv = ceil((tcnt[i + 1] - w) / NW): the sweeps stop there and read each
// vector's support as one contiguous prefix.  The entries past a support are
// exact zeros, so no sum changes.  T and m_pad = VPT T are compile-time
// constants, so the offsets of the values and of the vector slots are load
// immediates.
//
// Each Gram-Schmidt pass runs over the stored vectors in blocks of kGsBlock:
// one sweep forms the block's coefficients against the same w, one CTA
// reduction sums them, and one sweep subtracts them (block modified
// Gram-Schmidt; the vectors of a block are S-orthonormal, so within a block
// the coefficients equal those of the vector-by-vector order up to rounding,
// and the second pass removes what rounding leaves).  The update sweep
// re-reads the block's vectors, which the coefficient sweep has just brought
// into L2.  A reduction is a latency chain of shuffles, two barriers and the
// FP64 scalar work; blocks cut the chains per step from 2 (n + 1) + 1 to
// 2 ceil((n + 1) / kGsBlock) + 1.
//
// w lives in registers for small VPT and in shared memory for large; u
// (with its lo word in mixed precision) in shared memory when it fits, else
// re-read from global memory (an L2 hit: the SpMM has just written it).  In
// mixed precision the lo word of u only corrects h_{i,n} by about 2^-24
// relative, so its products are summed with plain FMAs and folded into the lo
// word of the accurate sum.
constexpr int kGsBlock = 4;

template <typename VT, int VPT, int T>
struct MgsCfg {
    static constexpr bool kLo = sizeof(VT) == 4;                    // u as (hi, lo) pair
    static constexpr bool kWs = VPT >= (sizeof(VT) == 4 ? 8 : 4);    // w in smem
    static constexpr bool kUs = kLo || !kWs || 2 * VPT * T * sizeof(VT) <= 160 * 1024;
    // values per batch of loads: pass-1 coefficients (8 streams), beta and
    // pass-2 coefficients (2 or 4 streams), subtractions (4 streams); FP64
    // is bound by its arithmetic and runs one value at a time
    static constexpr int kChunkDot = sizeof(VT) == 8 ? 1 : 2;
    static constexpr int kChunkSmall = sizeof(VT) == 8 ? 1 : 4;
    static constexpr int kChunkUpd = sizeof(VT) == 8 ? 1 : 4;
    static constexpr int kSmemVectors = (kUs ? 1 : 0) + (kLo ? 1 : 0) + (kWs ? 1 : 0);
};

// Live values of warp `warp` when the first cnt tile positions are live.
template <int T>
__device__ __forceinline__ int live_values(int cnt, int warp)
{
    constexpr int NW = T / 32;
    return cnt > warp ? (cnt - warp + NW - 1) / NW : 0;
}

// f(v, live) over the thread's first nv values, chunk by chunk; a compiler
// barrier between chunks keeps one chunk's loads live at a time, and only the
// last live chunk tests its values.
template <int VPT, int kChunk, typename F>
__device__ __forceinline__ void for_live(int nv, F &&f)
{
#pragma unroll
    for (int v0 = 0; v0 < VPT; v0 += kChunk) {
        if (v0 >= nv) break;
        if (v0 + kChunk <= nv) {
#pragma unroll
            for (int q = 0; q < kChunk && v0 + q < VPT; ++q) f(v0 + q, true);
        } else {
#pragma unroll
            for (int q = 0; q < kChunk && v0 + q < VPT; ++q) f(v0 + q, v0 + q < nv);
        }
        if (v0 + kChunk < VPT) asm volatile("" ::: "memory");
    }
}

// Sum of N per-thread accumulators over the CTA in a fixed order.  In each
// warp a reduce-scatter butterfly leaves value q = lane / (32 / N) on lanes
// q (32 / N) .. (q + 1) (32 / N) - 1 (each lane sends half of its values per
// round, so N values cost about as many shuffles as two), warp q then sums
// value q over the warps, and its lane 0 runs epi(q, total): the scalar FP64
// work of a reduction (scales, coefficients, the breakdown test) is done once
// there and handed to the CTA through shared memory.  `buf` alternates the
// partial slots so that two barriers per reduction suffice.
template <typename VT, int N, typename Epi>
__device__ __forceinline__ void block_sum(DotAcc<VT> (&a)[N], double *part, int &buf, Epi epi)
{
    static_assert(N == 1 || N == 2 || N == 4 || N == 8, "N must be 1, 2, 4 or 8");
    constexpr int LOGN = N == 8 ? 3 : N == 4 ? 2 : N == 2 ? 1 : 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
    for (int r = 0; r < LOGN; ++r) {
        const int o = 16 >> r, half = N >> (r + 1);
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            DotAcc<VT> keep = up ? a[j + half] : a[j];
            const DotAcc<VT> send = up ? a[j] : a[j + half];
            keep.merge(send.shfl_xor(o));
            a[j] = keep;
        }
    }
#pragma unroll
    for (int o = 16 >> LOGN; o > 0; o >>= 1) a[0].merge(a[0].shfl_xor(o));
    if ((lane & ((32 >> LOGN) - 1)) == 0) part[(buf * N + (lane >> (5 - LOGN))) * 32 + warp] = a[0].pack();
    __syncthreads();
    if (warp < N) {
        DotAcc<VT> x;
        if (lane < nw) x.unpack(part[(buf * N + warp) * 32 + lane]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x.merge(x.shfl_xor(o));
        if (lane == 0) epi(warp, x.value());
    }
    __syncthreads();
    buf ^= 1;
}

template <typename VT, int VPT, int T>
__global__ void __launch_bounds__(T, T == 256 ? 4 : T == 512 ? 2 : 1) mgs_kernel(
    VT *__restrict__ K, VT *__restrict__ SK, const VT *__restrict__ U, const VT *__restrict__ Ulo,
    double *__restrict__ Hsub, double *__restrict__ scale, double *__restrict__ cn2,
    int *__restrict__ status, int *__restrict__ nu_eff, const int *__restrict__ tcnt, int n, int nu,
    int need_w, double tau2)
{
    using Cfg = MgsCfg<VT, VPT, T>;
    constexpr bool kWs = Cfg::kWs, kUs = Cfg::kUs, kLo = Cfg::kLo;
    constexpr int kB = kGsBlock;
    constexpr int64_t MP = (int64_t)VPT * T;   // m_pad
    const int c = blockIdx.x;
    if (status[c] != 0) return;
    const int tid = threadIdx.x, warp = tid >> 5;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT *us = reinterpret_cast<VT *>(smem_raw);             // u = H w_n, unscaled (if kUs)
    VT *uls = us + (kUs ? MP : 0);                          // its lo word (mixed precision)
    VT *ws = uls + (kLo ? MP : 0);                          // w (if kWs)
    __shared__ double red[2 * 2 * kGsBlock * 32];   // reduction partials, two slots
    __shared__ double ctot[kMaxNu];
    __shared__ double ssc[kMaxNu];
    __shared__ int cnt_s[kMaxNu + 2];
    __shared__ VT coef[2][kGsBlock];   // FP32/FP64 update coefficients of the last reduction
    __shared__ double bc_sn;
    __shared__ int bc_stop;
    const int64_t base = (int64_t)c * nu * MP;
    int buf = 0;
    auto live = [&](int cnt) { return live_values<T>(cnt, warp); };

    for (int i = tid; i < n; i += T) ssc[i] = scale[(int64_t)c * nu + i];
    for (int L = tid; L <= n + 1; L += T) cnt_s[L] = tcnt[(int64_t)c * (nu + 2) + L];
    __syncthreads();

    // beta_n = ||w_n||_S and the breakdown test (slot 0 is stored normalised)
    double sn = 1.0;
    if (n > 0) {
        const VT *wn = K + base + (int64_t)n * MP + tid;
        const VT *swn = SK + base + (int64_t)n * MP + tid;
        DotAcc<VT> acc[1];
        for_live<VPT, Cfg::kChunkSmall>(live(cnt_s[n]), [&](int v, bool a) {
            acc[0].add(a ? wn[v * T] : VT(0), a ? swn[v * T] : VT(0));
        });
        block_sum(acc, red, buf, [&](int, double beta2) {
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
    // w starts as u = s_n H w_n; the h dots use H w_n unscaled (with its lo
    // word in mixed precision) and apply s_i s_n in FP64 after the reduction.
    // Positions past u's support hold zeros, which partly live chunks read.
    const VT vsn = (VT)sn;
    const VT *u = U + (int64_t)c * MP + tid;
    const VT *ul = kLo ? Ulo + (int64_t)c * MP + tid : nullptr;
    VT wr[kWs ? 1 : VPT];
    {
        const int nv = live(cnt_s[n + 1]);
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int p = tid + v * T;
            const bool a = v < nv;
            const VT x = a ? u[v * T] : VT(0);
            if constexpr (kWs) ws[p] = x * vsn; else wr[v] = x * vsn;
            if constexpr (kUs) us[p] = x;
            if constexpr (kLo) uls[p] = a ? ul[v * T] : VT(0);
        }
    }
    auto wget = [&](int v) -> VT {
        if constexpr (kWs) return ws[tid + v * T]; else return wr[v];
    };
    auto wset = [&](int v, VT x) {
        if constexpr (kWs) ws[tid + v * T] = x; else wr[v] = x;
    };
    // w -= sum_l coef_l k_{i0+l} over the block (vectors re-read from L2)
    auto update = [&](const VT *kb, const int (&nvl)[kB], int nvmax, const VT (&co)[kB]) {
        for_live<VPT, Cfg::kChunkUpd>(nvmax, [&](int v, bool a) {
            VT x = wget(v);
#pragma unroll
            for (int l = 0; l < kB; ++l) {
                const VT kr = (a && v < nvl[l]) ? kb[l * MP + v * T] : VT(0);
                x = fma(-co[l], kr, x);
            }
            wset(v, x);
        });
    };
    // pass 1: h_{i,n} = k_i . u and the first Gram-Schmidt sweep
    for (int i0 = 0; i0 <= n; i0 += kB) {
        const int nbk = min(kB, n + 1 - i0);
        int nvl[kB];
        int nvmax = 0;
#pragma unroll
        for (int l = 0; l < kB; ++l) {
            nvl[l] = l < nbk ? live(cnt_s[i0 + l + 1]) : 0;
            nvmax = max(nvmax, nvl[l]);
        }
        const VT *kb = K + base + (int64_t)i0 * MP + tid;
        const VT *skb = SK + base + (int64_t)i0 * MP + tid;
        DotAcc<VT> acc[2 * kB];   // [l]: c = S k . w, [kB + l]: h = k . u
        VT hl[kB];
#pragma unroll
        for (int l = 0; l < kB; ++l) hl[l] = VT(0);
        for_live<VPT, Cfg::kChunkDot>(nvmax, [&](int v, bool a) {
            const int p = tid + v * T;
            VT uu;
            if constexpr (kUs) uu = us[p]; else uu = a ? u[v * T] : VT(0);
            const VT wv = wget(v);
#pragma unroll
            for (int l = 0; l < kB; ++l) {
                const bool al = a && v < nvl[l];
                const VT kr = al ? kb[l * MP + v * T] : VT(0);
                acc[kB + l].add(kr, uu);
                if constexpr (kLo) hl[l] = fma(kr, uls[p], hl[l]);
                if (need_w) acc[l].add(al ? skb[l * MP + v * T] : VT(0), wv);
            }
        });
#pragma unroll
        for (int l = 0; l < kB; ++l) {
            if constexpr (kLo) acc[kB + l].add_lo(hl[l]);
        }
        block_sum(acc, red, buf, [&](int q, double t) {
            const int l = q < kB ? q : q - kB, i = i0 + l;
            if (l >= nbk) {
                if (q < kB) coef[buf][q] = VT(0);
                return;
            }
            const double si = i == n ? sn : ssc[i];
            if (q < kB) {
                const double ci = t * si;
                ctot[i] = ci;
                coef[buf][q] = (VT)(ci * si);
            } else {
                const double h = t * si * sn;
                Hsub[((int64_t)c * nu + i) * nu + n] = h;
                Hsub[((int64_t)c * nu + n) * nu + i] = h;
            }
        });
        if (need_w) {
            VT co[kB];
#pragma unroll
            for (int l = 0; l < kB; ++l) co[l] = coef[buf ^ 1][l];
            update(kb, nvl, nvmax, co);
        }
    }
    if (!need_w) return;
    // pass 2: second Gram-Schmidt sweep
    for (int i0 = 0; i0 <= n; i0 += kB) {
        const int nbk = min(kB, n + 1 - i0);
        int nvl[kB];
        int nvmax = 0;
#pragma unroll
        for (int l = 0; l < kB; ++l) {
            nvl[l] = l < nbk ? live(cnt_s[i0 + l + 1]) : 0;
            nvmax = max(nvmax, nvl[l]);
        }
        const VT *kb = K + base + (int64_t)i0 * MP + tid;
        const VT *skb = SK + base + (int64_t)i0 * MP + tid;
        DotAcc<VT> acc[kB];
        for_live<VPT, Cfg::kChunkSmall>(nvmax, [&](int v, bool a) {
            const VT wv = wget(v);
#pragma unroll
            for (int l = 0; l < kB; ++l)
                acc[l].add((a && v < nvl[l]) ? skb[l * MP + v * T] : VT(0), wv);
        });
        block_sum(acc, red, buf, [&](int q, double t) {
            if (q >= nbk) {
                coef[buf][q] = VT(0);
                return;
            }
            const int i = i0 + q;
            const double si = i == n ? sn : ssc[i];
            const double ci = t * si;
            ctot[i] += ci;
            coef[buf][q] = (VT)(ci * si);
        });
        VT co[kB];
#pragma unroll
        for (int l = 0; l < kB; ++l) co[l] = coef[buf ^ 1][l];
        update(kb, nvl, nvmax, co);
    }
    VT *wo = K + base + (int64_t)(n + 1) * MP + tid;   // the next slot, unnormalised, zeros included
#pragma unroll
    for (int v = 0; v < VPT; ++v) wo[v * T] = wget(v);
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
    if (b.shape.m_pad != (int64_t)VPT * T || b.ntile != VPT * T / 32 || !b.tcnt)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)VPT * T * sizeof(VT) * Cfg::kSmemVectors;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(mgs_kernel<VT, VPT, T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    mgs_kernel<VT, VPT, T><<<b.nb, T, smem, s>>>(
        (VT *)b.K, (VT *)b.SK, (const VT *)b.U, (const VT *)b.Ulo, b.Hsub, b.scale, b.cn2,
        b.status, b.nu_eff, b.tcnt, n, b.nu, need_w, tau * tau);
    return cudaGetLastError();
}

template <typename VT>
cudaError_t mgs_shape(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s)
{
    if (b.shape.threads == 512) {   // FP32, 16 values per thread
        if constexpr (sizeof(VT) == 4)
            if (b.shape.vpt == 16) return mgs_dispatch<VT, 16, 512>(b, n, need_w, tau, s);
        return cudaErrorInvalidValue;
    }
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
                                                 b.shape.m_pad, b.tinv, b.nb);
    else
        init_kernel<float><<<b.nb, 256, 0, s>>>(A.rp, A.ci, A.Sd, A.sdiag, b.cols, (float *)b.K,
                                                (float *)b.SK, b.scale, b.status, b.nu_eff, b.nu,
                                                b.shape.m_pad, b.tinv, b.nb);
    return cudaGetLastError();
}

cudaError_t launch_spmm_hs(const DeviceMatrix &A, const KrylovBatch &b, const void *X, int64_t ldx,
                           void *SY, int64_t ldsy, int lim, cudaStream_t s)
{
    if (!b.thop || !b.tinv || b.ntile * 8 < A.nbr) return cudaErrorInvalidValue;
    const dim3 block(32, 8);
    const dim3 grid((unsigned)((A.nbr + 7) / 8), (unsigned)((b.nb + 63) / 64));
    const int64_t ldu = b.shape.m_pad;
    if (b.prec == 0) {
        if (SY)
            spmm_hs_kernel<double, true><<<grid, block, 0, s>>>(
                A.nbr, A.rp, A.ci, A.Hd, A.Sd, (const double *)X, ldx, (double *)b.U, nullptr, ldu,
                (double *)SY, ldsy, b.nb, b.thop, b.tinv, lim);
        else
            spmm_hs_kernel<double, false><<<grid, block, 0, s>>>(
                A.nbr, A.rp, A.ci, A.Hd, A.Sd, (const double *)X, ldx, (double *)b.U, nullptr, ldu,
                nullptr, 0, b.nb, b.thop, b.tinv, lim);
    } else {
        if (SY)
            spmm_hs_kernel<float, true><<<grid, block, 0, s>>>(
                A.nbr, A.rp, A.ci, A.Hf, A.Sf, (const float *)X, ldx, (float *)b.U, (float *)b.Ulo, ldu,
                (float *)SY, ldsy, b.nb, b.thop, b.tinv, lim);
        else
            spmm_hs_kernel<float, false><<<grid, block, 0, s>>>(
                A.nbr, A.rp, A.ci, A.Hf, A.Sf, (const float *)X, ldx, (float *)b.U, (float *)b.Ulo, ldu,
                nullptr, 0, b.nb, b.thop, b.tinv, lim);
    }
    return cudaGetLastError();
}

cudaError_t launch_mgs(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s)
{
    return b.prec == 0 ? mgs_shape<double>(b, n, need_w, tau, s) : mgs_shape<float>(b, n, need_w, tau, s);
}

}  // namespace marnoldi
