// Device helpers shared by the Gram-Schmidt kernels (krylov.cu, gs_stream.cu):
// error-free FP32 dot accumulators, fixed-order CTA reductions, and the FP64
// scalar step of one Krylov step (norm, breakdown test, the Gram matrix's new
// column, the new row of L^-1 and the projection coefficients).
#pragma once

#include "internal.h"

namespace marnoldi {
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


// Two FP32 lanes per instruction (add/sub/mul/fma .rn.f32x2, sm_100 and
// later): each lane is rounded exactly as the scalar instruction would be, so
// a pair of independent sums runs at half the instruction count.  The pairs
// are formed and split inside the PTX (mov.b64 of two 32-bit registers), so
// that the register allocator can keep them as register pairs.
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 a, b, c, d;\n\t"
        "mov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\tmov.b64 c, {%6, %7};\n\t"
        "fma.rn.f32x2 d, a, b, c;\n\t"
        "mov.b64 {%0, %1}, d;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// Two DotAcc<float> side by side (lane x and lane y), updated with packed
// instructions: per lane the operations of DotAcc<float>::add (p = a b,
// e = fma(a, b, -p), the two-sum of hi and p, lo += e + err).
struct DotAcc2 {
    float2 hi = make_float2(0.f, 0.f), lo = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add(float2 a, float2 b)
    {
        asm("{\n\t.reg .b64 a, b, p, np, e, h, l, s, bb, t, u, err;\n\t"
            "mov.b64 a, {%4, %5};\n\tmov.b64 b, {%6, %7};\n\t"
            "mov.b64 h, {%0, %1};\n\tmov.b64 l, {%2, %3};\n\t"
            "mul.rn.f32x2 p, a, b;\n\t"
            "xor.b64 np, p, 0x8000000080000000;\n\t"
            "fma.rn.f32x2 e, a, b, np;\n\t"
            "add.rn.f32x2 s, h, p;\n\t"
            "sub.rn.f32x2 bb, s, h;\n\t"
            "sub.rn.f32x2 t, s, bb;\n\t"
            "sub.rn.f32x2 t, h, t;\n\t"
            "sub.rn.f32x2 u, p, bb;\n\t"
            "add.rn.f32x2 err, t, u;\n\t"
            "add.rn.f32x2 e, e, err;\n\t"
            "add.rn.f32x2 l, l, e;\n\t"
            "mov.b64 {%0, %1}, s;\n\tmov.b64 {%2, %3}, l;\n\t}"
            : "+f"(hi.x), "+f"(hi.y), "+f"(lo.x), "+f"(lo.y)
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    }
    __device__ __forceinline__ DotAcc<float> lane(int q) const
    {
        DotAcc<float> r;
        r.hi = q ? hi.y : hi.x;
        r.lo = q ? lo.y : lo.x;
        return r;
    }
};

// Two adjacent FP32 values as one 64-bit register (lane x = the lower
// address), and the packed (f32x2) operations on such pairs; each lane is
// rounded exactly as the scalar instruction would be.
__device__ __forceinline__ uint64_t lds2(const float *p)
{
    uint64_t r;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)));
    return r;
}
__device__ __forceinline__ uint64_t pair_of(float x)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ uint64_t fma_x2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ float lane_x(uint64_t a) { return __uint_as_float((unsigned)a); }
__device__ __forceinline__ float lane_y(uint64_t a) { return __uint_as_float((unsigned)(a >> 32)); }

// Two DotAcc<float> (one per lane) in packed registers: per lane the
// operations of DotAcc<float>::add (p = a b, e = fma(a, b, -p), the two-sum
// of hi and p, lo += e + err).
struct PairAcc {
    uint64_t hi = 0, lo = 0;
    __device__ __forceinline__ void add(uint64_t a, uint64_t b)
    {
        asm("{\n\t.reg .b64 p, np, e, s, bb, t, u, err;\n\t"
            "mul.rn.f32x2 p, %2, %3;\n\t"
            "xor.b64 np, p, 0x8000000080000000;\n\t"
            "fma.rn.f32x2 e, %2, %3, np;\n\t"
            "add.rn.f32x2 s, %0, p;\n\t"
            "sub.rn.f32x2 bb, s, %0;\n\t"
            "sub.rn.f32x2 t, s, bb;\n\t"
            "sub.rn.f32x2 t, %0, t;\n\t"
            "sub.rn.f32x2 u, p, bb;\n\t"
            "add.rn.f32x2 err, t, u;\n\t"
            "add.rn.f32x2 e, e, err;\n\t"
            "add.rn.f32x2 %1, %1, e;\n\t"
            "mov.b64 %0, s;\n\t}"
            : "+l"(hi), "+l"(lo)
            : "l"(a), "l"(b));
    }
    // the two lanes' sums, joined by a two-sum
    __device__ __forceinline__ DotAcc<float> joined() const
    {
        DotAcc<float> r;
        r.hi = lane_x(hi);
        r.lo = lane_x(lo);
        DotAcc<float> y;
        y.hi = lane_y(hi);
        y.lo = lane_y(lo);
        r.merge(y);
        return r;
    }
};

// Vectors per block of the Gram-Schmidt sweeps (one CTA reduction each).
constexpr int kGsBlock = 4;

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

// Barrier of a group of the CTA's threads: 0 = the whole CTA, else the named
// barrier `bar` over `nthreads` threads (whole warps).
__device__ __forceinline__ void group_sync(int bar, int nthreads)
{
    if (bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthreads) : "memory");
}

// Sum of N <= 16 per-thread accumulators over a group of warps (the CTA, or
// one of its halves) in a fixed order.  In each warp a reduce-scatter
// butterfly over NP = 2^ceil(log2 N) slots leaves slot q on lanes
// q (32 / NP) .. (q + 1) (32 / NP) - 1 (each lane sends half of its slots per
// round, so N values cost about as many shuffles as two); then warp w of the
// group sums values w, w + gnw, ... over its warps and its lane 0 runs
// epi(q, total).  `buf` alternates the partial slots (part holds
// 2 x 16 x stride doubles, stride >= gnw) so that two barriers per reduction
// suffice; `bar` selects the group's barrier (0: the CTA's).
// The warp step of block_sum: a reduce-scatter butterfly over NP =
// 2^ceil(log2 N) slots; slot q (q < N) ends, summed over the warp, on lanes
// q (32 / NP) .. (q + 1) (32 / NP) - 1 (each lane sends half of its slots per
// round, so N values cost about as many shuffles as two).  Returns the lane's
// slot total.
template <typename VT, int N>
__device__ __forceinline__ DotAcc<VT> warp_scatter(const DotAcc<VT> (&in)[N])
{
    static_assert(N >= 1 && N <= 16, "1 <= N <= 16");
    constexpr int LOGN = N > 8 ? 4 : N > 4 ? 3 : N > 2 ? 2 : N > 1 ? 1 : 0;
    constexpr int NP = 1 << LOGN;
    const int lane = threadIdx.x & 31;
    DotAcc<VT> a[NP];
#pragma unroll
    for (int q = 0; q < N; ++q) a[q] = in[q];
#pragma unroll
    for (int r = 0; r < LOGN; ++r) {
        const int o = 16 >> r, half = NP >> (r + 1);
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
    return a[0];
}

// Sum of N <= 16 per-thread accumulators over a group of warps (the CTA, or
// one of its halves) in a fixed order: warp_scatter in each warp, then warp w
// of the group sums values w, w + gnw, ... over its warps and its lane 0 runs
// epi(q, total).  `buf` alternates the partial slots (part holds
// 2 x 16 x stride doubles, stride >= gnw) so that two barriers per reduction
// suffice; `bar` selects the group's barrier (0: the CTA's).
template <typename VT, int N, typename Epi>
__device__ __forceinline__ void block_sum(const DotAcc<VT> (&in)[N], double *part, int &buf, Epi epi,
                                          int gwarp, int gnw, int stride, int bar)
{
    constexpr int LOGN = N > 8 ? 4 : N > 4 ? 3 : N > 2 ? 2 : N > 1 ? 1 : 0;
    const int lane = threadIdx.x & 31;
    const DotAcc<VT> a0 = warp_scatter(in);
    const int qm = lane >> (5 - LOGN);
    if ((lane & ((32 >> LOGN) - 1)) == 0 && qm < N) part[(buf * 16 + qm) * stride + gwarp] = a0.pack();
    group_sync(bar, gnw * 32);
    for (int q = gwarp; q < N; q += gnw) {
        DotAcc<VT> x;
        if (lane < gnw) x.unpack(part[(buf * 16 + q) * stride + lane]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x.merge(x.shfl_xor(o));
        if (lane == 0) epi(q, x.value());
    }
    group_sync(bar, gnw * 32);
    buf ^= 1;
}

// sum over the warp of x (every lane holds the total)
__device__ __forceinline__ double warp_total(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// Shared-memory arrays of the scalar step (length >= nu each).
template <typename VT>
struct GsScalarSmem {
    double *ssc;    // s_i (i < n) in, s_n set here
    double *ta;     // sweep totals a_i = w_i . u
    double *tb;     // b_i = (S w_i) . u
    double *tg;     // g_i = (S w_i) . w_n
    double *lrow;   // L^-1 G_{<n, n}
    double *nrow;   // the new row n of L^-1
    double *zc;     // L^-1 p
    VT *coef;       // subtraction coefficients c_i s_i
    int &stop;
    double &dinv;
};

// The FP64 scalar step of Krylov step n for column c, run by the T threads
// (thread index tid) that `sync` synchronises, after the sweep's totals are in
// ta, tb, tg: beta_n and the breakdown test, s_n, G's column n and the entries
// h_{m,n} of unit-norm vectors (into Hsub), the new row of L^-1 (into Lsub),
// and, when need_w, the coefficients c = L^-T L^-1 p of s_n u into coef and
// |L^-1 p|^2 into cn2[c].  Returns true when the subtraction w_{n+1} = s_n u -
// sum coef_i w_i follows (false: the column stopped, or the last step).  Lsub
// holds L^-1 (lower triangular), so every product is a matrix-vector product,
// one warp per row or column, with no serial chain.
template <typename VT, int T, typename Sync>
__device__ __forceinline__ bool gs_scalars(int c, int n, int nu, int need_w, double tau2, int tid,
                                           double *__restrict__ Hsub, double *__restrict__ Lsub,
                                           double *__restrict__ scale, double *__restrict__ cn2,
                                           int *__restrict__ status, int *__restrict__ nu_eff,
                                           GsScalarSmem<VT> sm, Sync sync)
{
    const int warp = tid >> 5, lane = tid & 31;
    double *Lc = Lsub + (int64_t)c * nu * nu;   // L^-1, row-major, lower triangle
    if (tid == 0) {
        double sn = 1.0;   // slot 0 is stored normalised (G_00 = 1)
        int stop = 0;
        if (n > 0) {
            const double beta2 = sm.tg[n];
            if (!(beta2 > 0.0) || beta2 <= tau2 * (beta2 + cn2[c])) {
                stop = 1;
                // a square norm below zero by no more than the threshold times the
                // projected part is rounding at breakdown (FP32 vectors near linear
                // dependence); further below, or NaN, it is not a norm (2)
                status[c] = (beta2 >= -sqrt(tau2) * cn2[c]) ? 1 : 2;
                nu_eff[c] = n;
            } else {
                sn = 1.0 / sqrt(beta2);
                scale[(int64_t)c * nu + n] = sn;
            }
        }
        sm.ssc[n] = sn;
        sm.stop = stop;
    }
    sync();
    if (sm.stop) return false;
    const double sn = sm.ssc[n];
    for (int m = tid; m <= n; m += T) {   // G_{mn}, p_m (of s_n u) and h_m of unit-norm vectors
        const double f = sm.ssc[m] * sn;
        sm.tg[m] *= f;
        sm.tb[m] *= f;
        const double h = sm.ta[m] * f;
        Hsub[((int64_t)c * nu + m) * nu + n] = h;
        Hsub[((int64_t)c * nu + n) * nu + m] = h;
    }
    sync();
    constexpr int NW = T / 32;
    // l = L^-1 G_{<n, n}
    for (int r = warp; r < n; r += NW) {
        double x = 0.0;
        for (int m = lane; m <= r; m += 32) x = fma(Lc[(int64_t)r * nu + m], sm.tg[m], x);
        x = warp_total(x);
        if (lane == 0) sm.lrow[r] = x;
    }
    sync();
    // d = sqrt(G_nn - |l|^2), G_nn = 1; the new row of L^-1 is (-l^T L^-1, 1) / d
    if (warp == 0) {
        double x = 0.0;
        for (int r = lane; r < n; r += 32) x = fma(sm.lrow[r], sm.lrow[r], x);
        x = warp_total(x);
        if (lane == 0) {
            const double dd = 1.0 - x;
            if (!(dd > 0.0)) {   // the stored basis has lost its rank
                sm.stop = 1;
                status[c] = 1;
                nu_eff[c] = n;
            } else {
                sm.dinv = 1.0 / sqrt(dd);
            }
        }
    }
    sync();
    if (sm.stop) return false;
    const double dinv = sm.dinv;
    double *Ln = Lc + (int64_t)n * nu;
    for (int m = warp; m < n; m += NW) {
        double x = 0.0;
        for (int r = m + lane; r < n; r += 32) x = fma(sm.lrow[r], Lc[(int64_t)r * nu + m], x);
        x = warp_total(x);
        if (lane == 0) {
            sm.nrow[m] = -dinv * x;
            Ln[m] = -dinv * x;
        }
    }
    if (tid == 0) {
        sm.nrow[n] = dinv;
        Ln[n] = dinv;
    }
    sync();
    if (!need_w) return false;
    // z = L^-1 p, |z|^2 = |projection of s_n u|_S^2, c = L^-T z
    for (int r = warp; r <= n; r += NW) {
        const double *Lr = r == n ? sm.nrow : Lc + (int64_t)r * nu;
        double x = 0.0;
        for (int m = lane; m <= r; m += 32) x = fma(Lr[m], sm.tb[m], x);
        x = warp_total(x);
        if (lane == 0) sm.zc[r] = x;
    }
    sync();
    for (int m = warp; m <= n; m += NW) {
        double x = 0.0;
        for (int r = m + lane; r <= n; r += 32) x = fma(r == n ? sm.nrow[m] : Lc[(int64_t)r * nu + m], sm.zc[r], x);
        x = warp_total(x);
        if (lane == 0) sm.coef[m] = (VT)(x * sm.ssc[m]);
    }
    if (warp == 0) {
        double x = 0.0;
        for (int r = lane; r <= n; r += 32) x = fma(sm.zc[r], sm.zc[r], x);
        x = warp_total(x);
        if (lane == 0) cn2[c] = x;
    }
    sync();
    return true;
}

}  // namespace
}  // namespace marnoldi
