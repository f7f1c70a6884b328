// Krylov-subspace build of the multiple Arnoldi method on sm_103a.
//
// For a batch of columns j, builds a basis of
// span{e_j, H e_j, ..., H^(nu-1) e_j} (arXiv:1307.3218, Section 2: the subspace
// L_nu^(j) containing e_j whose nu x nu *standard* eigenproblem replaces
// H phi = eps S phi, Eq. 2), its S-Gram matrix and the explicit subspace
// matrix of the stored vectors; the eigensolve turns them into the
// S-orthonormal basis K and H_sub = K^T H K.
//
// The basis is stored unnormalised: slot i holds w_i and S w_i, and
// k_i = s_i w_i with s_i = 1 / ||w_i||_S.  One Krylov step n, for every column:
//   spmm_hs:  H w_n into U (accurate (hi, lo) in mixed precision) and, for
//             n >= 1, S w_n into slot n (one gather of w_n for both)
//   gs:       beta_n^2 = w_n . S w_n; stop the column when
//             beta_n^2 <= tau^2 (beta_n^2 + |projection of u_{n-1}|_S^2), i.e.
//             ||w_n||_S <= tau ||u_{n-1}||_S; else s_n = 1 / beta_n, the
//             entries k_i . H k_n, the Gram column k_i . S k_n, and
//             w_{n+1} = s_n H w_n - (its S-projection on span(K)) into slot n+1
//
// Inner products are accumulated to FP64 accuracy where the result needs it;
// in mixed precision the vectors, the SpMM and the Gram-Schmidt updates are
// FP32.  Reductions use a fixed order (warp butterflies, then one warp over
// the warps), so results do not depend on scheduling.
#include "gs_common.cuh"

#include <cstdio>

namespace marnoldi {

const char *kernel_name(int kind)
{
    static const char *names[KK_NKINDS] = {"init",   "spmm_H", "gs",      "spmm_S", "eigsub",
                                           "minmax", "count",  "density", "green", "region", "support", "spmm_HS",
                                           "bisect_step", "force", "eigenstate"};
    return (kind >= 0 && kind < KK_NKINDS) ? names[kind] : "?";
}

// Vectors up to 4096 entries run 256-thread CTAs (several columns share an SM
// and overlap each other's reductions).  Longer FP32 vectors up to 8192
// entries run 512-thread CTAs of 16 values per thread (two per SM); longer
// FP32 vectors run the streamed kernel (gs_stream.cu) with 256 consumer
// threads of 64 values and a producer warp, two CTAs per SM (shape {64, 288};
// {32, 544}, one CTA of 512 consumer threads per SM, is the other streamed
// shape); the rest run 1024-thread CTAs.  VPT is the power of two that covers m.
ColumnShape column_shape(int64_t m, int prec)
{
    if (prec == 1 && m > 4096 && m <= 8192) return ColumnShape{16, 512, 8192};
    if (prec == 1 && m > 8192 && m <= 16384) return ColumnShape{64, 288, 16384};   // gs_stream.cu
    const int T = m <= 4096 ? 256 : 1024;
    int v = 1;
    while (v < 16 && (int64_t)v * T < m) v *= 2;
    return ColumnShape{v, T, (int64_t)v * T};
}

int column_shape_candidates(int64_t m_pad, int prec, ColumnShape *out)
{
    int n = 0;
    for (int T : {256, 512, 1024})
        for (int v = 1; v <= 16; v *= 2)
            if ((int64_t)v * T == m_pad) out[n++] = ColumnShape{v, T, m_pad};
    for (const ColumnShape st : {ColumnShape{32, 544, 16384}, ColumnShape{64, 288, 16384}})
        if (m_pad == st.m_pad && gs_stream_shape(st, prec)) out[n++] = st;
    return n;
}

namespace {

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
        for (int a = 0; a < 4; ++a) {
            const int64_t q = vpos(tinv, nb, c, 4 * I + a);
            if (in_range(q, m_pad, kChkInitPos)) sk0[q] = (VT)(Sv[16 * k + 4 * b + a] * inv);
        }
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
            if (L[0].act) {
                const int64_t xp = 4 * apos(tinv, ncols, cc[0], J);
                if (in_range(xp, ldu - 3, kChkSpmmGather)) load4(x0 + xp, xv[0]);
            }
            if (L[1].act) {
                const int64_t xp = 4 * apos(tinv, ncols, cc[1], J);
                if (in_range(xp, ldu - 3, kChkSpmmGather)) load4(x1 + xp, xv[1]);
            }
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
        // rows outside the support get their zeros, except rows of another
        // structure of a union, whose tiles may sit past this column's positions
        if (!L[h].live || yo[h] >= ldu) continue;
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

// ------------------------------------------------------------------ Gram-Schmidt
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
// Orthogonalisation (one pass, with the exact S-Gram matrix).  The stored
// vectors w_i, scaled to unit S-norm (k_i = s_i w_i), are S-orthonormal only
// up to rounding; their Gram matrix G = K^T S K = L L^T is kept exactly
// through L^-1 (its new row every step from G's new column), so that every
// solve with G is a pair of matrix-vector products.  Step n
// forms, in one sweep over the stored vectors i <= n (blocks of kGsBlock
// vectors, one CTA reduction each),
//   a_i = w_i . u          H_sub entries of the stored basis (u = H w_n)
//   b_i = (S w_i) . u      right-hand side of the S-projection of u
//   g_i = (S w_i) . w_n    G's column n (g_n = beta_n^2)
// then, in FP64 over the CTA, the S-projection coefficients c = G^-1 p of
// s_n u onto span(K) and subtracts them in a streaming sweep with no
// reductions: w_{n+1} = s_n u - sum_i c_i k_i.  Whatever rounding leaves
// along span(K) is carried by G, so the subspace problem, solved on
// L^-1 H_sub L^-T, is the exact Rayleigh-Ritz projection on the stored
// vectors.  The subspace is span{e_j, H e_j, ...} whatever the coefficients,
// so in exact arithmetic this is the method's Arnoldi basis; per stored vector
// and step it reads w_i and S w_i once for the coefficients and w_i once for
// the subtraction (three vector reads, against four for two Gram-Schmidt
// passes), and runs one reduction per block instead of two.
//
// In mixed precision a_i and g_i are accumulated error-free (exact FP32
// products, two-sums, (hi, lo) pairs; the lo word of u, which only corrects
// a_i by about 2^-24, through plain FMAs).  b_i is summed per thread with
// plain FMAs (the CTA reduction stays accurate): its rounding only leaves a
// component of w_{n+1} along span(K) at the level the FP32 subtraction leaves
// anyway, which G records.  The coefficients and G are FP64.
// u (and its lo word) and w sit in shared memory (or registers for small
// VPT); w holds w_n during the coefficient sweep and w_{n+1} afterwards.
template <typename VT, int VPT, int T>
struct GsCfg {
    static constexpr bool kLo = sizeof(VT) == 4;                    // u as (hi, lo) pair
    static constexpr bool kWs = VPT >= (sizeof(VT) == 4 ? 8 : 4);    // w in smem
    static constexpr bool kUs = kLo || !kWs || 2 * VPT * T * sizeof(VT) <= 160 * 1024;
    static constexpr int kChunkDot = sizeof(VT) == 8 ? 1 : 2;        // values per batch of loads
    static constexpr int kChunkUpd = sizeof(VT) == 8 ? 1 : 4;
    static constexpr int kSmemVectors = (kUs ? 1 : 0) + (kLo ? 1 : 0) + (kWs ? 1 : 0);
};

template <typename VT, int VPT, int T>
__global__ void __launch_bounds__(T, T == 256 ? 4 : T == 512 ? 2 : 1) gs_kernel(
    VT *__restrict__ K, VT *__restrict__ SK, const VT *__restrict__ U, const VT *__restrict__ Ulo,
    double *__restrict__ Hsub, double *__restrict__ Lsub, double *__restrict__ scale,
    double *__restrict__ cn2, int *__restrict__ status, int *__restrict__ nu_eff,
    const int *__restrict__ tcnt, int n, int nu, int need_w, double tau2)
{
    using Cfg = GsCfg<VT, VPT, T>;
    constexpr bool kWs = Cfg::kWs, kUs = Cfg::kUs, kLo = Cfg::kLo;
    constexpr int kB = kGsBlock;
    constexpr int64_t MP = (int64_t)VPT * T;   // m_pad
    const int c = blockIdx.x;
    if (status[c] != 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    VT *us = reinterpret_cast<VT *>(smem_raw);             // u = H w_n, unscaled (if kUs)
    VT *uls = us + (kUs ? MP : 0);                          // its lo word (mixed precision)
    VT *ws = uls + (kLo ? MP : 0);                          // w_n, then w_{n+1} (if kWs)
    __shared__ double red[2 * 16 * 32];   // reduction partials, two slots
    __shared__ double ssc[kMaxNu];        // s_i, then s_n
    __shared__ double ta[kMaxNu], tb[kMaxNu], tg[kMaxNu];   // the sweep's totals
    __shared__ double lrow[kMaxNu];       // L^-1 G_{<n, n}
    __shared__ double nrow[kMaxNu];       // the new row n of L^-1
    __shared__ double zc[kMaxNu];         // L^-1 p
    __shared__ int cnt_s[kMaxNu + 2];
    __shared__ VT coef[kMaxNu];           // subtraction coefficients c_i s_i
    __shared__ int bc_stop;
    __shared__ double bc_dinv;
    const int64_t base = (int64_t)c * nu * MP;
    int buf = 0;
    auto live = [&](int cnt) { return live_values<T>(cnt, warp); };

    for (int i = tid; i < n; i += T) ssc[i] = scale[(int64_t)c * nu + i];
    for (int L = tid; L <= n + 1; L += T) {
        const int t = tcnt[(int64_t)c * (nu + 2) + L];
        cnt_s[L] = in_range(t, MP / 32 + 1, kChkSupportCount) ? t : (int)(MP / 32);
    }
    __syncthreads();

    // u (hi, lo) and w_n on chip; zeros past their supports
    const VT *u = U + (int64_t)c * MP + tid;
    const VT *ul = kLo ? Ulo + (int64_t)c * MP + tid : nullptr;
    const VT *wnp = K + base + (int64_t)n * MP + tid;
    VT wr[kWs ? 1 : VPT];
    auto wget = [&](int v) -> VT {
        if constexpr (kWs) return ws[tid + v * T]; else return wr[v];
    };
    auto wset = [&](int v, VT x) {
        if constexpr (kWs) ws[tid + v * T] = x; else wr[v] = x;
    };
    {
        const int nvu = live(cnt_s[n + 1]), nvn = live(cnt_s[n]);
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int p = tid + v * T;
            const bool a = v < nvu;
            if constexpr (kUs) us[p] = a ? u[v * T] : VT(0);
            if constexpr (kLo) uls[p] = a ? ul[v * T] : VT(0);
            wset(v, v < nvn ? wnp[v * T] : VT(0));
        }
    }
    auto block_live = [&](int i0, int nbk, int (&nvl)[kB]) {
        int m = 0;
#pragma unroll
        for (int l = 0; l < kB; ++l) {
            nvl[l] = l < nbk ? live(cnt_s[i0 + l + 1]) : 0;
            m = max(m, nvl[l]);
        }
        return m;
    };

    // ---- coefficient sweep over the stored vectors i <= n.  With G = 2 the
    // CTA's halves take alternate blocks of vectors, each over all entries
    // (thread t of a half owns positions t + v T/2), and reduce on their own
    // barriers, so that one half's loads overlap the other's reduction.  This
    // pays for FP64 vectors (6 % on a 16,384-entry sweep); FP32 vectors, whose
    // error-free sums need more registers, ran slower with it (spills, or
    // fewer loads in flight) and keep one group.
    constexpr int G = (sizeof(VT) == 8 && T == 1024 && kWs && VPT >= 8) ? 2 : 1;
    constexpr int TG = T / G, VG = VPT * G;
    const int grp = tid / TG, gtid = tid - grp * TG, gwarp = gtid >> 5;
    double *gpart = red + grp * (2 * 16 * 32 / G);
    const VT *ug = U + (int64_t)c * MP + gtid;
    auto glive = [&](int cnt) { return live_values<TG>(cnt, gwarp); };
    if constexpr (G > 1) __syncthreads();   // u and w_n were stored by other threads
    for (int i0 = grp * kB; i0 <= n; i0 += G * kB) {
        const int nbk = min(kB, n + 1 - i0);
        int nvl[kB];
        int nvmax = 0;
#pragma unroll
        for (int l = 0; l < kB; ++l) {
            nvl[l] = l < nbk ? glive(cnt_s[i0 + l + 1]) : 0;
            nvmax = max(nvmax, nvl[l]);
        }
        const VT *kb = K + base + (int64_t)i0 * MP + gtid;
        const VT *skb = SK + base + (int64_t)i0 * MP + gtid;
        DotAcc<VT> acc[3 * kB];   // [l] a, [kB + l] b, [2 kB + l] g
        VT hl[kB], bp[kB];
#pragma unroll
        for (int l = 0; l < kB; ++l) hl[l] = bp[l] = VT(0);
        for_live<VG, Cfg::kChunkDot>(nvmax, [&](int v, bool a) {
            const int p = gtid + v * TG;
            VT uu;
            if constexpr (kUs) uu = us[p]; else uu = a ? ug[v * TG] : VT(0);
            VT wn;
            if constexpr (G > 1) wn = ws[p]; else wn = wget(v);
#pragma unroll
            for (int l = 0; l < kB; ++l) {
                const bool al = a && v < nvl[l];
                const VT kr = al ? kb[l * MP + v * TG] : VT(0);
                const VT sr = al ? skb[l * MP + v * TG] : VT(0);
                acc[l].add(kr, uu);
                if constexpr (kLo) hl[l] = fma(kr, uls[p], hl[l]);
                if (need_w) bp[l] = fma(sr, uu, bp[l]);
                acc[2 * kB + l].add(sr, wn);
            }
        });
#pragma unroll
        for (int l = 0; l < kB; ++l) {
            if constexpr (kLo) acc[l].add_lo(hl[l]);
            acc[kB + l].set(bp[l]);
        }
        block_sum(acc, gpart, buf, [&](int q, double t) {
            const int l = q % kB, i = i0 + l;
            if (l >= nbk) return;
            if (q < kB) ta[i] = t; else if (q < 2 * kB) tb[i] = t; else tg[i] = t;
        }, gwarp, TG / 32, 32 / G, G > 1 ? 1 + grp : 0);
    }
    if constexpr (G > 1) __syncthreads();   // both halves' totals

    // ---- scalars, G's column, the new row of L^-1, the coefficients (FP64).
    // Lc holds L^-1 (lower triangular), so every product below is a matrix-
    // vector product, one warp per row or column, with no serial chain.
    {
        const GsScalarSmem<VT> sm{ssc, ta, tb, tg, lrow, nrow, zc, coef, bc_stop, bc_dinv};
        if (!gs_scalars<VT, T>(c, n, nu, need_w, tau2, tid, Hsub, Lsub, scale, cn2, status, nu_eff, sm,
                               [] { __syncthreads(); }))
            return;
    }

    // ---- w_{n+1} = s_n u - sum_i coef_i w_i: streaming subtraction, last block
    // first (its vectors are the ones the sweep read last; its support is u's)
    const VT vsn = (VT)ssc[n];
    const int nb1 = (n + kB) / kB;
    for (int b = nb1 - 1; b >= 0; --b) {
        const int i0 = b * kB, nbk = min(kB, n + 1 - i0);
        int nvl[kB];
        const int nvmax = block_live(i0, nbk, nvl);
        const bool first = b == nb1 - 1;
        const int nvs = first ? live(cnt_s[n + 1]) : nvmax;
        const VT *kb = K + base + (int64_t)i0 * MP + tid;
        VT co[kB];
#pragma unroll
        for (int l = 0; l < kB; ++l) co[l] = l < nbk ? coef[i0 + l] : VT(0);
        for_live<VPT, Cfg::kChunkUpd>(nvs, [&](int v, bool a) {
            if constexpr (kLo) {
                // FP32 vectors: the sum runs as a (hi, lo) pair (hi in w's
                // place, lo in u's lo word, which is no longer needed), with
                // exact products and two-sums, and is rounded to FP32 once
                // at the end: s_n u and the projection nearly cancel, so a
                // plain FP32 chain would leave rounding errors of the size of
                // s_n u, not of w_{n+1}, outside span(K)
                const int p = tid + v * T;
                DotAcc<VT> x;
                if (first) {
                    x.add(vsn, us[p]);
                    x.lo = __fmaf_rn(vsn, uls[p], x.lo);
                } else {
                    x.hi = wget(v);
                    x.lo = uls[p];
                }
#pragma unroll
                for (int l = 0; l < kB; ++l)
                    x.add(-co[l], (a && v < nvl[l]) ? kb[l * MP + v * T] : VT(0));
                wset(v, x.hi);
                uls[p] = x.lo;
            } else {
                VT x;
                if (first) {
                    VT uu;
                    if constexpr (kUs) uu = us[tid + v * T]; else uu = a ? u[v * T] : VT(0);
                    x = uu * vsn;
                } else {
                    x = wget(v);
                }
#pragma unroll
                for (int l = 0; l < kB; ++l)
                    x = fma(-co[l], (a && v < nvl[l]) ? kb[l * MP + v * T] : VT(0), x);
                wset(v, x);
            }
        });
    }
    VT *wo = K + base + (int64_t)(n + 1) * MP + tid;   // the next slot, unnormalised, zeros included
    const int nvu = live(cnt_s[n + 1]);
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        VT x = VT(0);
        if (v < nvu) {
            if constexpr (kLo) x = __fadd_rn(wget(v), uls[tid + v * T]); else x = wget(v);
        }
        wo[v * T] = x;
    }
}

template <typename VT, int VPT, int T>
cudaError_t gs_dispatch(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s)
{
    using Cfg = GsCfg<VT, VPT, T>;
    if (b.shape.m_pad != (int64_t)VPT * T || (int64_t)b.ntile * 32 < b.shape.m_pad || !b.tcnt || !b.Lsub)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)VPT * T * sizeof(VT) * Cfg::kSmemVectors;
    cudaError_t e = allow_dynamic_smem((const void *)gs_kernel<VT, VPT, T>, smem);
    if (e != cudaSuccess) return e;
    gs_kernel<VT, VPT, T><<<b.nb, T, smem, s>>>(
        (VT *)b.K, (VT *)b.SK, (const VT *)b.U, (const VT *)b.Ulo, b.Hsub, b.Lsub, b.scale, b.cn2,
        b.status, b.nu_eff, b.tcnt, n, b.nu, need_w, tau * tau);
    return cudaGetLastError();
}

template <typename VT, int T>
cudaError_t gs_vpt(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s)
{
    switch (b.shape.vpt) {
    case 1: return gs_dispatch<VT, 1, T>(b, n, need_w, tau, s);
    case 2: return gs_dispatch<VT, 2, T>(b, n, need_w, tau, s);
    case 4: return gs_dispatch<VT, 4, T>(b, n, need_w, tau, s);
    case 8: return gs_dispatch<VT, 8, T>(b, n, need_w, tau, s);
    case 16: return gs_dispatch<VT, 16, T>(b, n, need_w, tau, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename VT>
cudaError_t gs_shape(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s)
{
    switch (b.shape.threads) {
    case 256: return gs_vpt<VT, 256>(b, n, need_w, tau, s);
    case 512: return gs_vpt<VT, 512>(b, n, need_w, tau, s);
    case 1024: return gs_vpt<VT, 1024>(b, n, need_w, tau, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

MARNOLDI_CHECK_TAKE(krylov)

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

cudaError_t launch_gs(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s)
{
    if (gs_stream_shape(b.shape, b.prec)) return launch_gs_stream(b, n, need_w, tau, s);
    return b.prec == 0 ? gs_shape<double>(b, n, need_w, tau, s) : gs_shape<float>(b, n, need_w, tau, s);
}

}  // namespace marnoldi
