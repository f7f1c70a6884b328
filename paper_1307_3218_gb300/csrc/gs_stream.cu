// Gram-Schmidt step of the Krylov build with the stored vectors streamed
// through a shared-memory ring by the bulk-copy (TMA) engine, for FP32 Krylov
// vectors of 16,384 entries (mixed precision, global mode on structures of
// 2,049 to 4,096 atoms).
//
// It computes what gs_kernel (krylov.cu) computes for one Krylov step n of one
// column (arXiv:1307.3218, Section 2: the S-orthonormal basis of the Krylov
// subspace L_nu^(j) and its subspace matrix): the sweep totals
//   a_i = w_i . u,  b_i = (S w_i) . u,  g_i = (S w_i) . w_n   (i <= n, u = H w_n)
// in blocks of four stored vectors, the FP64 scalar step (gs_scalars), and the
// subtraction w_{n+1} = s_n u - sum_i c_i s_i w_i (a (hi, lo) sum, rounded
// to FP32 once).  The arithmetic per value is the same; the values are
// grouped differently over the threads, so results agree with gs_kernel's
// shapes to rounding.
//
// What differs is how the vectors reach the arithmetic.  gs_kernel loads them
// with the CTA's own threads, so its loads and its reductions alternate in
// step and HBM idles during every block reduction.  Here a producer warp
// feeds a ring of R slots; a slot holds one chunk (2 T entries, T / 16 tiles
// of 32, for T consumer threads) of the four vectors w_i and the four S w_i
// of a block and of u = H w_n, its lo word and w_n, copied by cp.async.bulk
// straight from each vector's support prefix (the vectors are stored in the
// column's hop order, so a support is one contiguous prefix) and signalled on
// the slot's "full" mbarrier with the bytes it carries.  The consumer warps
// wait on "full", compute, and release the slot on its "empty" mbarrier (one
// arrival per warp); the producer refills a slot once it is empty, so copies of later
// chunks stay in flight while the consumers finish a block and while they
// run the scalar step.  A consumer thread takes two adjacent entries of each
// vector with one 64-bit shared-memory load and runs both through one packed
// FP32 instruction (f32x2), which halves the instruction count of the
// error-free arithmetic.  The block sums need no CTA barrier: the last warp
// to finish a block adds up the warps' partial sums.  u, its lo word and w_n
// come again with every block (from L2: they are the column's most recently
// used data), so the ring takes all the dynamic shared memory.  The
// subtraction runs chunk by chunk: for each chunk the blocks' w_i, last block
// first, with u, each value's (hi, lo) sum in registers and stored once its
// chunk is done.
//
// Shapes: 512 consumer threads with a ring of 4 slots of 11 pieces of 1,024
// floats (176 KB, one CTA per SM), or 256 consumer threads with 3 slots of 11
// pieces of 512 floats (66 KB, two CTAs per SM).
//
// Every wait is bounded: an mbarrier wait gives up after kWaitLimitNs of the
// global timer, sets the CTA's abort flag (later waits then return at once, so
// the CTA runs to its end through the same barriers) and the column's status
// to 3; the host reports MARNOLDI_ETIMEOUT.
#include "gs_common.cuh"

namespace marnoldi {
namespace {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s per wait

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// One bulk copy global -> shared (16-byte aligned addresses, bytes a multiple
// of 16), completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// The same copy with an L2 eviction-priority hint (a policy from createpolicy).
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                              uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_last_policy()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Wait until phase `parity` of `bar` has completed.  Bounded: false once the
// CTA's abort flag is set, or after kWaitLimitNs (which sets it).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = 0;
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*abort) return false;
            const unsigned long long t = global_ns();
            if (t0 == 0) {
                t0 = t;
            } else if (t - t0 > kWaitLimitNs) {
                *abort = 1;
                return false;
            }
        }
    }
}

// Wait at most ns nanoseconds for phase `parity` of `bar`.
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t parity, unsigned long long ns)
{
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > ns) return false;
    return true;
}

__device__ __forceinline__ void named_sync(int bar, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthreads) : "memory");
}

// Live tiles (32 entries) of chunk v (tiles NW v .. NW v + NW - 1) of a vector
// whose support is its first cnt tiles.
template <int NW>
__device__ __forceinline__ int chunk_tiles(int cnt, int v)
{
    return max(0, min(NW, cnt - NW * v));
}

// Ring slot layout (floats, CH = 2 T per piece): w_{i0+l} at 2 l CH,
// S w_{i0+l} at (2 l + 1) CH (l < 4), u at 8 CH, its lo word at 9 CH and w_n at
// 10 CH, each the chunk of positions v CH .. v CH + CH - 1 (only the live
// tiles are copied).
constexpr int kSlotPieces = 2 * kGsBlock + 3;
constexpr int64_t kStreamM = 16384;             // vector length (m_pad)

// Dynamic shared memory of the kernel below: the ring of R slots.
template <int T, int R>
constexpr size_t gs_stream_smem()
{
    return (size_t)R * kSlotPieces * 2 * T * sizeof(float);
}

// T consumer threads (NW = T / 32 warps); warp NW is the producer; R ring
// slots; MINB CTAs share an SM (two, when the ring and the scalar arrays fit
// in half of shared memory, so that one CTA's block sums and scalar step
// overlap the other's copies).  A chunk v
// is positions v CH .. v CH + CH - 1 (CH = 2 T = 32 NW, tiles 32 v .. 32 v + 31);
// thread tid takes positions v CH + 2 tid and + 1 (tile 32 v + tid / 16), as a
// pair in one 64-bit register, and the two lanes of the packed instructions are
// these two positions.
//
// Stages, in the order both sides take them:
//   coefficient sweep: for each block b of four stored vectors, each chunk v
//     that holds live tiles of the block: w_i, S w_i (i in b), u, u lo, w_n
//   subtraction: for each chunk v of u's support, each pair of blocks b, b - 1
//     (last first) that hold live tiles in chunk v: w_i (i in b and b - 1),
//     and u, u lo with the last block.  The first R of them are copied
//     before the scalar step
//     (when a subtraction follows at all: need_w), and the consumers drain
//     them if the column stops there.
//
// Block sums without a CTA barrier: at the end of a block each warp joins its
// lanes, reduces the 12 sums over its threads (warp_scatter) and stores them in
// the block's partial buffer; the warp that arrives last (a ticket in shared
// memory) adds the warps' partials in warp order and stores the totals.  A warp
// runs at most R stages (so R blocks) ahead of the slowest one, since a slot
// is refilled only when every warp has released it; R + 2 buffers, used in
// turn, are therefore never overwritten while read.
template <int T, int64_t MP, int R, int MINB>
__global__ void __launch_bounds__(T + 32, MINB) gs_stream_kernel(
    float *__restrict__ K, const float *__restrict__ SK, const float *__restrict__ U,
    const float *__restrict__ Ulo, double *__restrict__ Hsub, double *__restrict__ Lsub,
    double *__restrict__ scale, double *__restrict__ cn2, int *__restrict__ status,
    int *__restrict__ nu_eff, const int *__restrict__ tcnt, int n, int nu, int need_w, double tau2)
{
    constexpr int NW = T / 32;
    constexpr int CH = 2 * T;                 // positions per chunk
    constexpr int TPC = CH / 32;              // tiles per chunk
    constexpr int kB = kGsBlock;
    constexpr int SLOT = kSlotPieces * CH;    // floats per ring slot
    constexpr int kPartBufs = R + 2;          // per-block partial-sum buffers
    static_assert(MP % CH == 0, "whole chunks");
    const int c = blockIdx.x;
    if (status[c] != 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool producer = warp == NW;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>(smem_raw);
    __shared__ __align__(8) uint64_t full[R], empty[R];
    __shared__ double part[kPartBufs][3 * kB][NW];
    __shared__ int ticket[kPartBufs];
    __shared__ double ssc[kMaxNu];
    __shared__ double ta[kMaxNu], tb[kMaxNu], tg[kMaxNu];
    __shared__ double lrow[kMaxNu], nrow[kMaxNu], zc[kMaxNu];
    __shared__ int cnt_s[kMaxNu + 2];
    __shared__ float coef[kMaxNu];
    __shared__ int4 bcnt[kMaxNu / kGsBlock + 1];
    __shared__ float4 bcoef[kMaxNu / kGsBlock + 1];
    __shared__ int bch[kMaxNu / kGsBlock + 1];
    __shared__ int bc_stop, s_go, s_abort;
    __shared__ double bc_dinv;
    volatile int *abort = &s_abort;
    const int64_t base = (int64_t)c * nu * MP;

    for (int i = tid; i < n; i += T + 32) ssc[i] = scale[(int64_t)c * nu + i];
    for (int L = tid; L <= n + 1; L += T + 32) {
        const int t = tcnt[(int64_t)c * (nu + 2) + L];
        cnt_s[L] = in_range(t, MP / 32 + 1, kChkSupportCount) ? t : (int)(MP / 32);
    }
    if (tid < kPartBufs) ticket[tid] = 0;
    if (tid == T) {
        for (int s = 0; s < R; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        s_abort = 0;
        mbar_fence_init();
    }
    __syncthreads();
    const int cnt_u = cnt_s[n + 1];   // tiles of u's support (and of w_{n+1})
    const int cnt_n = cnt_s[n];       // tiles of w_n's support
    const int nb1 = (n + kB) / kB;    // blocks of stored vectors
    const int nch_u = (cnt_u + TPC - 1) / TPC;
    // chunks of block b (its last vector has the largest support)
    auto block_chunks = [&](int b) { return (cnt_s[min(b * kB + kB, n + 1)] + TPC - 1) / TPC; };
    // subtraction stages, and how many are copied ahead of the scalar step
    int nsub = 0;
    for (int v = 0; v < nch_u; ++v)
        for (int b = nb1 - 1; b >= 0 && block_chunks(b) > v; b -= 2) ++nsub;
    const int npre = need_w ? min(R, nsub) : 0;
    const float *ug = U + (int64_t)c * MP;
    const float *ulg = Ulo + (int64_t)c * MP;

    if (producer) {
        // ---- the producer warp
        uint32_t stage = 0;
        const uint64_t keep = l2_evict_last_policy();
        // one stage.  Coefficient sweep (sub = false): chunk v of block b's w_i
        // (piece 2 l) and S w_i (2 l + 1), of u (8), u lo (9) and w_n (10).
        // Subtraction (sub = true): chunk v of block b's w_i (piece 2 l) and,
        // when two, of block b - 1's (2 l + 1), with u and u lo when b is the
        // last block.  Lane q sizes piece q, lane 0 arms the slot's barrier
        // with their sum, then each lane copies its piece.
        auto issue = [&](int b, int v, bool sub, bool two) {
            const int s = (int)(stage % R);
            mbar_wait(&empty[s], ((stage / R) & 1) ^ 1, abort);
            const int64_t off = (int64_t)v * CH;
            const bool with_u = !sub || b == nb1 - 1;
            int vec = -1;      // the stored vector of piece `lane`, if any
            uint32_t bq = 0;
            const float *src = nullptr;
            if (lane < 8) {
                const int l = lane >> 1;
                const int bb = (sub && (lane & 1)) ? b - 1 : b;
                const bool used = sub ? (!(lane & 1) || two) : true;
                if (used && bb * kB + l <= n) vec = bb * kB + l;
                if (vec >= 0) {
                    bq = (uint32_t)chunk_tiles<TPC>(cnt_s[vec + 1], v) * 128u;
                    src = ((!sub && (lane & 1)) ? SK : K) + base + (int64_t)vec * MP + off;
                }
            } else if (lane < 10) {
                if (with_u) bq = (uint32_t)chunk_tiles<TPC>(cnt_u, v) * 128u;
                src = (lane == 8 ? ug : ulg) + off;
            } else if (lane == 10 && !sub) {
                bq = (uint32_t)chunk_tiles<TPC>(cnt_n, v) * 128u;
                src = K + base + (int64_t)n * MP + off;
            }
            const uint32_t bytes = __reduce_add_sync(0xffffffffu, bq);
            if (lane == 0) mbar_arrive_expect_tx(&full[s], bytes);
            __syncwarp();
            if (bq) {
                // u, its lo word and w_n come again with every block: keep them in L2
                if (lane >= 8) bulk_g2s_hint(ring + (int64_t)s * SLOT + (int64_t)lane * CH, src, bq, &full[s], keep);
                else bulk_g2s(ring + (int64_t)s * SLOT + (int64_t)lane * CH, src, bq, &full[s]);
            }
            __syncwarp();
            ++stage;
        };
        // subtraction stages with index in [from, to)
        auto subtraction = [&](int from, int to) {
            int k = 0;
            for (int v = 0; v < nch_u; ++v)
                for (int b = nb1 - 1; b >= 0 && block_chunks(b) > v; b -= 2, ++k)
                    if (k >= from && k < to) issue(b, v, true, b >= 1 && block_chunks(b - 1) > v);
        };
        for (int b = 0; b < nb1; ++b) {
            const int nch = block_chunks(b);
            for (int v = 0; v < nch; ++v) issue(b, v, false, false);
        }
        subtraction(0, npre);
        named_sync(2, T + 32);   // the consumers' scalar step is done
        if (s_go) subtraction(npre, nsub);
        return;
    }

    // ---- consumers: coefficient sweep
    uint32_t stage = 0;
    int slot = 0;              // stage % R
    uint32_t phase = 0;        // (stage / R) & 1
    auto next = [&] {
        ++stage;
        if (++slot == R) {
            slot = 0;
            phase ^= 1u;
        }
    };
    const int ktile = tid >> 4;   // this thread's tile within a chunk
    for (int b = 0; b < nb1; ++b) {
        const int i0 = b * kB, nbk = min(kB, n + 1 - i0);
        const int nch = block_chunks(b);
        int cl[kB];
#pragma unroll
        for (int l = 0; l < kB; ++l) cl[l] = l < nbk ? cnt_s[i0 + l + 1] : 0;
        PairAcc pa[kB], pg[kB];
        uint64_t hl[kB], bp[kB];
#pragma unroll
        for (int l = 0; l < kB; ++l) hl[l] = bp[l] = 0;
        for (int v = 0; v < nch; ++v) {
            mbar_wait(&full[slot], phase, abort);
            const int k = TPC * v + ktile;
            const float *sl = ring + (int64_t)slot * SLOT + 2 * tid;
            const uint64_t uu = k < cnt_u ? lds2(sl + 8 * CH) : 0;
            const uint64_t ul = k < cnt_u ? lds2(sl + 9 * CH) : 0;
            const uint64_t wn = k < cnt_n ? lds2(sl + 10 * CH) : 0;
#pragma unroll
            for (int l = 0; l < kB; ++l) {
                const bool al = k < cl[l];
                const uint64_t kr = al ? lds2(sl + 2 * l * CH) : 0;
                const uint64_t sr = al ? lds2(sl + (2 * l + 1) * CH) : 0;
                pa[l].add(kr, uu);
                hl[l] = fma_x2(kr, ul, hl[l]);
                if (need_w) bp[l] = fma_x2(sr, uu, bp[l]);
                pg[l].add(sr, wn);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
            next();
        }
        DotAcc<float> acc[3 * kB];   // [l] a, [kB + l] b, [2 kB + l] g
#pragma unroll
        for (int l = 0; l < kB; ++l) {
            acc[l] = pa[l].joined();
            acc[l].add_lo(__fadd_rn(lane_x(hl[l]), lane_y(hl[l])));
            acc[kB + l].set(__fadd_rn(lane_x(bp[l]), lane_y(bp[l])));
            acc[2 * kB + l] = pg[l].joined();
        }
        // the warp's sums into the block's buffer; the last warp adds them up
        constexpr int N = 3 * kB;
        constexpr int LOGN = 4;   // N = 12 slots in 16
        const DotAcc<float> a0 = warp_scatter(acc);
        const int qm = lane >> (5 - LOGN);
        const int pb = b % kPartBufs;
        if ((lane & ((32 >> LOGN) - 1)) == 0 && qm < N) part[pb][qm][warp] = a0.pack();
        __threadfence_block();
        __syncwarp();
        int last = 0;
        if (lane == 0) last = atomicAdd(&ticket[pb], 1) == NW - 1;
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            __threadfence_block();
            if (lane < N) {
                DotAcc<float> x;
                x.unpack(part[pb][lane][0]);
                for (int w = 1; w < NW; ++w) {
                    DotAcc<float> y;
                    y.unpack(part[pb][lane][w]);
                    x.merge(y);
                }
                const int l = lane % kB, i = i0 + l;
                if (l < nbk) {
                    const double t = x.value();
                    if (lane < kB) ta[i] = t; else if (lane < 2 * kB) tb[i] = t; else tg[i] = t;
                }
            }
            if (lane == 0) atomicExch(&ticket[pb], 0);
        }
    }
    named_sync(1, T);   // every block's totals are stored

    // ---- the FP64 scalar step over the consumer threads, then meet the producer
    const GsScalarSmem<float> sm{ssc, ta, tb, tg, lrow, nrow, zc, coef, bc_stop, bc_dinv};
    const bool go = gs_scalars<float, T>(c, n, nu, need_w, tau2, tid, Hsub, Lsub, scale, cn2, status, nu_eff,
                                         sm, [] { named_sync(1, T); });
    if (tid == 0) s_go = go ? 1 : 0;
    named_sync(2, T + 32);
    if (!go) {
        // the column stopped: let the stages copied ahead land before exit
        for (int q = 0; q < npre; ++q) {
            mbar_wait(&full[slot], phase, abort);
            next();
        }
    } else {
        // ---- w_{n+1} = s_n u - sum_i coef_i w_i, chunk by chunk; per value
        // the blocks last first, as a (hi, lo) sum with exact products and
        // two-sums, rounded to FP32 once (s_n u and the projection nearly
        // cancel: a plain FP32 chain would leave rounding errors of the size
        // of s_n u, not of w_{n+1}, outside span(K))
        const uint64_t vsn = pair_of((float)ssc[n]);
        float *wo = K + base + (int64_t)(n + 1) * MP;   // the next slot, zeros included
        // per block: its vectors' live tiles and -coefficients (0 past the
        // block's last vector), and its chunk count
        for (int b = tid; b < nb1; b += T) {
            const int i0 = b * kB, nbk = min(kB, n + 1 - i0);
            int cn[kB];
            float cf[kB];
#pragma unroll
            for (int l = 0; l < kB; ++l) {
                cn[l] = l < nbk ? cnt_s[i0 + l + 1] : 0;
                cf[l] = l < nbk ? -coef[i0 + l] : 0.f;
            }
            bcnt[b] = make_int4(cn[0], cn[1], cn[2], cn[3]);
            bcoef[b] = make_float4(cf[0], cf[1], cf[2], cf[3]);
            bch[b] = block_chunks(b);
        }
        named_sync(1, T);
        for (int v = 0; v < nch_u; ++v) {
            const int k = TPC * v + ktile;
            PairAcc x;
            for (int b = nb1 - 1; b >= 0 && bch[b] > v; b -= 2) {
                mbar_wait(&full[slot], phase, abort);
                const float *sl = ring + (int64_t)slot * SLOT + 2 * tid;
                if (b == nb1 - 1) {
                    const bool a = k < cnt_u;
                    x.add(vsn, a ? lds2(sl + 8 * CH) : 0);
                    x.lo = fma_x2(vsn, a ? lds2(sl + 9 * CH) : 0, x.lo);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {   // block b (even pieces), then block b - 1 (odd)
                    const int bb = b - h;
                    if (h == 1 && (bb < 0 || bch[bb] <= v)) break;
                    const int4 cn = bcnt[bb];
                    const float4 cf = bcoef[bb];
                    x.add(k < cn.x ? pair_of(cf.x) : 0, k < cn.x ? lds2(sl + h * CH) : 0);
                    x.add(k < cn.y ? pair_of(cf.y) : 0, k < cn.y ? lds2(sl + (2 + h) * CH) : 0);
                    x.add(k < cn.z ? pair_of(cf.z) : 0, k < cn.z ? lds2(sl + (4 + h) * CH) : 0);
                    x.add(k < cn.w ? pair_of(cf.w) : 0, k < cn.w ? lds2(sl + (6 + h) * CH) : 0);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                next();
            }
            const int64_t p = (int64_t)v * CH + 2 * tid;
            const float2 r = k < cnt_u ? make_float2(__fadd_rn(lane_x(x.hi), lane_x(x.lo)),
                                                     __fadd_rn(lane_y(x.hi), lane_y(x.lo)))
                                       : make_float2(0.f, 0.f);
            *reinterpret_cast<float2 *>(wo + p) = r;
        }
        for (int64_t p = (int64_t)nch_u * CH + 2 * tid; p < MP; p += CH)
            *reinterpret_cast<float2 *>(wo + p) = make_float2(0.f, 0.f);
    }
    if (*abort) {
        // a wait gave up: give the copies that may still be in flight into
        // shared memory a bounded time to land before the CTA's shared memory
        // is released (the next phase of each slot's "full" barrier), and flag
        // the column
        if (tid == 0) {
            for (int s = 0; s < R; ++s) {
                const uint32_t uses = stage > (uint32_t)s ? (stage - (uint32_t)s + R - 1) / R : 0;
                mbar_wait_for(&full[s], uses & 1, 1000000ull);
            }
            status[c] = 3;
        }
    }
}

}  // namespace

// The two streamed shapes, as (values per consumer thread, threads per CTA):
// {32, 544}: 512 consumer threads and the producer, a ring of 4 slots of 44 KB,
// one CTA per SM; {64, 288}: 256 consumer threads and the producer, a ring of
// 3 slots of 22 KB, two CTAs per SM.
bool gs_stream_shape(const ColumnShape &s, int prec)
{
    return prec == 1 && s.m_pad == kStreamM &&
           ((s.vpt == 32 && s.threads == 544) || (s.vpt == 64 && s.threads == 288));
}

namespace {
template <int T, int R, int MINB>
cudaError_t launch_stream_shape(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s)
{
    constexpr int64_t MP = kStreamM;
    const size_t smem = gs_stream_smem<T, R>();
    cudaError_t e = allow_dynamic_smem((const void *)gs_stream_kernel<T, MP, R, MINB>, smem);
    if (e != cudaSuccess) return e;
    gs_stream_kernel<T, MP, R, MINB><<<b.nb, T + 32, smem, s>>>(
        (float *)b.K, (const float *)b.SK, (const float *)b.U, (const float *)b.Ulo, b.Hsub, b.Lsub, b.scale,
        b.cn2, b.status, b.nu_eff, b.tcnt, n, b.nu, need_w, tau * tau);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_gs_stream(const KrylovBatch &b, int n, int need_w, double tau, cudaStream_t s)
{
    if (!gs_stream_shape(b.shape, b.prec) || (int64_t)b.ntile * 32 < kStreamM || !b.tcnt || !b.Lsub || !b.Ulo)
        return cudaErrorInvalidValue;
    if (b.shape.threads == 288) return launch_stream_shape<256, 3, 2>(b, n, need_w, tau, s);
    return launch_stream_shape<512, 4, 1>(b, n, need_w, tau, s);
}

MARNOLDI_CHECK_TAKE(gs_stream)

}  // namespace marnoldi
