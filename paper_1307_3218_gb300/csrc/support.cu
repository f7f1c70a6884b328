// Structural support of the Krylov vectors of the multiple Arnoldi method.
//
// The subspace of column j is span{e_j, H e_j, ..., H^(nu-1) e_j}
// (arXiv:1307.3218, Section 2).  Its i-th basis vector is a combination of
// H^l e_j (l <= i), so it vanishes on every atom more than i hops from the
// column's atom J in the block pattern of H and S; S and H applied to it
// vanish beyond i + 1 hops.  The values there are exact zeros (sums of
// products with exact zeros), so a kernel that skips those entries computes
// bit for bit what the dense sweep computes.  Early basis vectors of a large
// cell cover a small part of it: on 4096-atom amorphous carbon at nu = 30 the
// Gram-Schmidt sweeps touch about two thirds of the dense entries.
//
// A structure may be a block-diagonal union of independent structures whose
// atom ranges start at multiples of 8 atoms: the search from J never leaves
// J's own structure, so only its tiles get the first positions and the
// vectors need only as many positions as the largest of them (tiles of the
// other structures sort behind and are never read or written).
//
// support_kernel: one CTA per batch column runs a breadth-first search from
// J over the block pattern (global mode) or the region's local pattern
// (regional mode), capped at nu + 1 hops, and summarises it per tile of 8
// atoms (32 vector entries): thop[t][c] (fewest hops into tile t), the
// position of each tile in (thop, t) order, and the number of tiles within
// each hop count.  The column's vectors are stored in that tile order, so
// every basis vector's support is a prefix of its slot.
#include "internal.h"

namespace marnoldi {
namespace {

template <bool kRegional>
__global__ void __launch_bounds__(256) support_kernel(
    const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, int nbr,
    const int *__restrict__ reg, int n_reg, int maxrow, const int *__restrict__ lcnt,
    const int *__restrict__ lci, const int64_t *__restrict__ cols, int nb, int ntile, int maxlev,
    int nlev, uint8_t *__restrict__ thop, uint16_t *__restrict__ tinv, int *__restrict__ tcnt)
{
    extern __shared__ uint8_t dist[];   // per atom (global or local index)
    __shared__ uint8_t th[kMaxTiles];
    __shared__ int start[256];
    const int c = blockIdx.x, tid = threadIdx.x;
    const int na = kRegional ? n_reg : nbr;
    const int Jg = (int)(cols[c] >> 2);
    const int J = kRegional ? find_sorted(reg + (int64_t)c * n_reg, n_reg, Jg) : Jg;
    const int64_t lbase = (int64_t)c * maxrow * n_reg;
    for (int a = tid; a < na; a += blockDim.x) dist[a] = a == J ? 0 : 255;
    __syncthreads();
    // level-synchronous search; every writer of dist[b] in a level writes the
    // same value, and a reader of the level's frontier never sees it change
    for (int lev = 0; lev < maxlev; ++lev) {
        int grew = 0;
        for (int a = tid; a < na; a += blockDim.x) {
            if (dist[a] != lev) continue;
            if constexpr (kRegional) {
                const int cnt = lcnt[(int64_t)c * n_reg + a];
                for (int s = 0; s < cnt; ++s) {
                    const int b = lci[lbase + (int64_t)s * n_reg + a];
                    if (dist[b] == 255) { dist[b] = (uint8_t)(lev + 1); grew = 1; }
                }
            } else {
                for (int64_t k = rp[a]; k < rp[a + 1]; ++k) {
                    const int b = ci[k];
                    if (dist[b] == 255) { dist[b] = (uint8_t)(lev + 1); grew = 1; }
                }
            }
        }
        if (!__syncthreads_or(grew)) break;
    }
    for (int t = tid; t < ntile; t += blockDim.x) {
        int h = 255;
        const int a1 = min(8 * t + 8, na);
        for (int a = 8 * t; a < a1; ++a) h = min(h, (int)dist[a]);
        th[t] = (uint8_t)h;
        thop[(int64_t)t * nb + c] = (uint8_t)h;
    }
    __syncthreads();
    if (tid == 0) {   // stable counting sort of the tiles by hop count
        for (int L = 0; L <= maxlev; ++L) start[L] = 0;
        for (int t = 0; t < ntile; ++t)
            if (th[t] <= maxlev) ++start[th[t]];
        int run = 0;
        for (int L = 0; L <= maxlev; ++L) {
            const int n = start[L];
            start[L] = run;
            run += n;
            tcnt[(int64_t)c * (nlev + 1) + L] = run;
        }
        for (int L = maxlev + 1; L <= nlev; ++L)   // past the search depth: every tile
            tcnt[(int64_t)c * (nlev + 1) + L] = ntile;
        int tail = run;
        for (int t = 0; t < ntile; ++t) {
            const int h = th[t];
            tinv[(int64_t)t * nb + c] = (uint16_t)(h <= maxlev ? start[h]++ : tail++);
        }
    }
}

// Rows past the last atom (or region atom) in its tile of 8 belong to no
// atom: the products never write them, so a later batch would read the
// previous batch's values there.  One CTA per batch column stores zeros at
// their positions in U (and its lo word) and in every S w slot (slot 0 is
// cleared by the initialisation, the K slots by every Gram-Schmidt writeout).
template <typename VT>
__global__ void zero_partial_tile_kernel(int rows, int nb, int nu, int64_t m_pad, const uint16_t *__restrict__ tinv,
                                         VT *__restrict__ SK, VT *__restrict__ U, VT *__restrict__ Ulo)
{
    const int c = blockIdx.x;
    const int r0 = rows, r1 = (rows + 7) & ~7;
    const int64_t base = 32 * (int64_t)tinv[(int64_t)(r0 >> 3) * nb + c];   // the tile's first entry
    if (base >= m_pad) return;   // a tile of another structure of a union: no position here
    const int nent = 4 * (r1 - r0);
    const int64_t e0 = base + 4 * (int64_t)(r0 & 7);
    for (int idx = threadIdx.x; idx < (nu + 1) * nent; idx += blockDim.x) {
        const int slot = idx / nent, e = idx - slot * nent;
        if (slot < nu) {
            if (slot > 0) SK[((int64_t)c * nu + slot) * m_pad + e0 + e] = VT(0);
        } else {
            U[(int64_t)c * m_pad + e0 + e] = VT(0);
            if (Ulo) Ulo[(int64_t)c * m_pad + e0 + e] = VT(0);
        }
    }
}

}  // namespace

cudaError_t launch_zero_partial_tile(const KrylovBatch &b, int rows, cudaStream_t s)
{
    if ((rows & 7) == 0 || b.nb < 1) return cudaSuccess;
    if (b.prec == 0)
        zero_partial_tile_kernel<double><<<b.nb, 128, 0, s>>>(rows, b.nb, b.nu, b.shape.m_pad, b.tinv, (double *)b.SK,
                                                              (double *)b.U, nullptr);
    else
        zero_partial_tile_kernel<float><<<b.nb, 128, 0, s>>>(rows, b.nb, b.nu, b.shape.m_pad, b.tinv, (float *)b.SK,
                                                             (float *)b.U, (float *)b.Ulo);
    return cudaGetLastError();
}

cudaError_t launch_support(const DeviceMatrix &A, const RegionMaps *rm, const KrylovBatch &b,
                           cudaStream_t s)
{
    // hop counts up to nu + 1 matter; a uint8 holds up to 254 of them (255 =
    // farther), and a tile beyond 254 hops is live for every level from 255 on
    const int nlev = b.nu + 1, maxlev = nlev < 254 ? nlev : 254;
    if (b.ntile > kMaxTiles || (int64_t)b.ntile * 32 < b.shape.m_pad) return cudaErrorInvalidValue;
    // more tiles than vector positions (a union of structures, each within
    // m_pad): only tiles within the search depth may get positions in use
    if ((int64_t)b.ntile * 32 > b.shape.m_pad && maxlev < nlev) return cudaErrorInvalidValue;
    if (rm) {
        if (rm->n_reg > kMaxRegion) return cudaErrorInvalidValue;
        support_kernel<true><<<b.nb, 256, rm->n_reg, s>>>(
            A.rp, A.ci, (int)A.nbr, rm->reg, rm->n_reg, rm->maxrow, rm->lcnt, rm->lci, b.cols, b.nb,
            b.ntile, maxlev, nlev, b.thop, b.tinv, b.tcnt);
    } else {
        if (A.nbr > kMaxGlobalM / 4) return cudaErrorInvalidValue;
        support_kernel<false><<<b.nb, 256, (size_t)A.nbr, s>>>(
            A.rp, A.ci, (int)A.nbr, nullptr, 0, 0, nullptr, nullptr, b.cols, b.nb, b.ntile, maxlev,
            nlev, b.thop, b.tinv, b.tcnt);
    }
    return cudaGetLastError();
}

}  // namespace marnoldi
