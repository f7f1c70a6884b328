// Regional (projection) mode of the multiple Arnoldi method on sm_103a.
//
// The method's cost is order-N (arXiv:1307.3218, Section 1): each column's
// Krylov process touches only a neighbourhood of its atom.  In regional mode
// the process for column j = 4 J + b runs on the principal sub-pair of (H, S)
// over J's projection region R_J: the n_reg atoms nearest J by squared
// minimum-image distance (ties to the lower atom index), kept in ascending
// atom index.  Local orbital 4 p + a is orbital a of atom R_J[p].
//
// Per batch column c (a region depends only on the column's atom, so of a
// run of batch columns of one atom only the first, its leader, searches):
//   region_kernel:     candidates from the cell list within radius r_s,
//                      bitonic sort by (d^2, index), the first n_reg sorted
//                      again by index -> reg[c][p]
//   local_bsr_kernel:  copies the leader's region to the other columns of
//                      its run; for every local block row p, the blocks of global row
//                      R_J[p] whose column atom lies in R_J (binary search):
//                      local column lci and global block index lgk, stored
//                      slot-major ([c][slot][p]) so that lanes over p coalesce
//   init_regional:     k_1 = e_{jl} / sqrt(S_jj), S k_1 from row j's local blocks
//   spmm_regional_hs:  H_local x and S_local x in one pass per group of one
//                      atom's columns (each block read once for the group),
//                      x and y of length m_pad >= 4 n_reg, matrix values
//                      gathered from the global BSR through lgk
#include "internal.h"

#include <cfloat>
#include <climits>

namespace marnoldi {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Squared minimum-image distance, summed as (dx^2 + dy^2) + dz^2 with every
// operation rounded separately (no contraction), so the host-side checker can
// reproduce the same values.
__device__ __forceinline__ double min_image_d2(const double *pi, const double *pj,
                                               const double *box)
{
    double d2 = 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double d = __dsub_rn(pi[q], pj[q]);
        d = __dsub_rn(d, __dmul_rn(box[q], rint(__ddiv_rn(d, box[q]))));
        d2 = q == 0 ? __dmul_rn(d, d) : __dadd_rn(d2, __dmul_rn(d, d));
    }
    return d2;
}

// First batch column of the run of consecutive batch columns that share
// column c's atom.
__device__ __forceinline__ int run_leader(const int64_t *__restrict__ cols, int c)
{
    const int64_t J = cols[c] >> 2;
    int l = c;
    while (l > 0 && (cols[l - 1] >> 2) == J) --l;
    return l;
}

__device__ __forceinline__ bool key_less(double da, int ia, double db, int ib)
{
    return da < db || (da == db && ia < ib);
}

// In-place bitonic sort of n (a power of two) (key, index) pairs in shared memory.
__device__ void bitonic_sort(double *key, int *idx, int n)
{
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
                const int lo = 2 * stride * (t / stride) + (t % stride);
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const bool sw = up ? key_less(key[hi], idx[hi], key[lo], idx[lo])
                                   : key_less(key[lo], idx[lo], key[hi], idx[hi]);
                if (sw) {
                    const double tk = key[lo]; key[lo] = key[hi]; key[hi] = tk;
                    const int ti = idx[lo]; idx[lo] = idx[hi]; idx[hi] = ti;
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(1024) region_kernel(
    const double *__restrict__ pos, const double *__restrict__ box,
    const int *__restrict__ cell_start, const int *__restrict__ cell_atoms, int3 ncell,
    double cell_edge_x, double cell_edge_y, double cell_edge_z, const int64_t *__restrict__ cols,
    int n_reg, double rs2, int hx, int hy, int hz, int cap, int *__restrict__ reg,
    int *__restrict__ rstat)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *key = reinterpret_cast<double *>(smem_raw);
    int *idx = reinterpret_cast<int *>(key + cap);
    __shared__ int count;
    __shared__ double bx[3], pj[3];
    const int c = blockIdx.x;
    const int J = (int)(cols[c] >> 2);
    if (c > 0 && (cols[c - 1] >> 2) == J) {   // not a leader: local_bsr_kernel copies the region
        if (threadIdx.x == 0) rstat[c] = 0;
        return;
    }
    if (threadIdx.x < 3) {
        bx[threadIdx.x] = box[threadIdx.x];
        pj[threadIdx.x] = pos[3 * (int64_t)J + threadIdx.x];
    }
    if (threadIdx.x == 0) count = 0;
    __syncthreads();
    const int cx = min(ncell.x - 1, max(0, (int)(pj[0] / cell_edge_x)));
    const int cy = min(ncell.y - 1, max(0, (int)(pj[1] / cell_edge_y)));
    const int cz = min(ncell.z - 1, max(0, (int)(pj[2] / cell_edge_z)));
    // distinct cells of the cube [c - h, c + h] (the whole axis when it wraps onto itself)
    const int nx = min(2 * hx + 1, ncell.x), ny = min(2 * hy + 1, ncell.y), nz = min(2 * hz + 1, ncell.z);
    const int ncube = nx * ny * nz;
    for (int q = threadIdx.x; q < ncube; q += blockDim.x) {   // one cell per thread
        const int ox = q % nx, oy = (q / nx) % ny, oz = q / (nx * ny);
        const int gx = ((nx == ncell.x ? ox : cx - hx + ox) % ncell.x + ncell.x) % ncell.x;
        const int gy = ((ny == ncell.y ? oy : cy - hy + oy) % ncell.y + ncell.y) % ncell.y;
        const int gz = ((nz == ncell.z ? oz : cz - hz + oz) % ncell.z + ncell.z) % ncell.z;
        const int cell = (gz * ncell.y + gy) * ncell.x + gx;
        for (int s = cell_start[cell]; s < cell_start[cell + 1]; ++s) {
            const int a = cell_atoms[s];
            const double d2 = min_image_d2(pos + 3 * (int64_t)a, pj, bx);
            if (d2 <= rs2) {
                const int slot = atomicAdd(&count, 1);
                if (slot < cap) {
                    key[slot] = d2;
                    idx[slot] = a;
                }
            }
        }
    }
    __syncthreads();
    const int cnt = count;
    if (cnt < n_reg || cnt > cap) {   // uniform: the host widens or narrows r_s and retries
        if (threadIdx.x == 0) rstat[c] = cnt < n_reg ? 1 : 2;
        return;
    }
    int n2 = 1;
    while (n2 < cnt) n2 <<= 1;
    for (int s = cnt + threadIdx.x; s < n2; s += blockDim.x) {
        key[s] = DBL_MAX;
        idx[s] = INT_MAX;
    }
    __syncthreads();
    bitonic_sort(key, idx, n2);
    // the n_reg nearest, again in ascending atom index: second sort with the
    // atom index as key (m2 <= n2 <= cap, cap a power of two)
    int m2 = 1;
    while (m2 < n_reg) m2 <<= 1;
    for (int s = threadIdx.x; s < m2; s += blockDim.x) {
        const bool in = s < n_reg;
        const int a = in ? idx[s] : INT_MAX;
        key[s] = in ? (double)a : DBL_MAX;
        idx[s] = a;
    }
    __syncthreads();
    bitonic_sort(key, idx, m2);
    for (int s = threadIdx.x; s < n_reg; s += blockDim.x) reg[(int64_t)c * n_reg + s] = idx[s];
    if (threadIdx.x == 0) rstat[c] = 0;
}

__global__ void __launch_bounds__(256) local_bsr_kernel(
    const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, const int64_t *__restrict__ cols,
    int *__restrict__ reg, int n_reg, int maxrow, int *__restrict__ lcnt, int *__restrict__ lci,
    int *__restrict__ lgk)
{
    const int c = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_reg) return;
    const int lead = run_leader(cols, c);
    const int *R = reg + (int64_t)lead * n_reg;
    const int I = R[p];
    if (lead != c) reg[(int64_t)c * n_reg + p] = I;
    int cnt = 0;
    const int64_t base = (int64_t)c * maxrow * n_reg;
    for (int64_t k = rp[I]; k < rp[I + 1]; ++k) {
        const int q = find_sorted(R, n_reg, ci[k]);
        if (q >= 0) {
            lci[base + (int64_t)cnt * n_reg + p] = q;
            lgk[base + (int64_t)cnt * n_reg + p] = (int)k;
            ++cnt;
        }
    }
    lcnt[(int64_t)c * n_reg + p] = cnt;
}

// k_1 = e_{jl} / sqrt(S_jj) and S k_1 from row j's local blocks (S symmetric).
template <typename VT>
__global__ void init_regional_kernel(const double *__restrict__ Sv, const double *__restrict__ sdiag,
                                     const int64_t *__restrict__ cols, const int *__restrict__ reg,
                                     int n_reg, int maxrow, const int *__restrict__ lcnt,
                                     const int *__restrict__ lci, const int *__restrict__ lgk,
                                     VT *__restrict__ K, VT *__restrict__ SK,
                                     double *__restrict__ scale, int *__restrict__ status,
                                     int *__restrict__ nu_eff, int nu, int64_t m_pad,
                                     const uint16_t *__restrict__ tinv, int nb)
{
    const int c = blockIdx.x;
    const int64_t j = cols[c];
    const int J = (int)(j >> 2), b = (int)(j & 3);
    VT *k0 = K + (int64_t)c * nu * m_pad;
    VT *sk0 = SK + (int64_t)c * nu * m_pad;
    for (int64_t r = threadIdx.x; r < m_pad; r += blockDim.x) {
        k0[r] = VT(0);
        sk0[r] = VT(0);
    }
    __syncthreads();
    // J is always inside its own region (distance 0); the guard only keeps the
    // writes in bounds should a region ever lack it (the column is then failed)
    const int pJ = find_sorted(reg + (int64_t)c * n_reg, n_reg, J);
    if (pJ < 0) {
        if (threadIdx.x == 0) {
            status[c] = 2;
            nu_eff[c] = 1;
        }
        return;
    }
    const double inv = 1.0 / sqrt(sdiag[j]);
    if (threadIdx.x == 0) {
        k0[vpos(tinv, nb, c, 4 * pJ + b)] = (VT)inv;
        scale[(int64_t)c * nu] = 1.0;
        status[c] = 0;
        nu_eff[c] = nu;
    }
    const int64_t base = (int64_t)c * maxrow * n_reg;
    const int cnt = lcnt[(int64_t)c * n_reg + pJ];
    for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
        const int q = lci[base + (int64_t)s * n_reg + pJ];
        const int64_t k = lgk[base + (int64_t)s * n_reg + pJ];
#pragma unroll
        for (int a = 0; a < 4; ++a) sk0[vpos(tinv, nb, c, 4 * q + a)] = (VT)(Sv[16 * k + 4 * b + a] * inv);
    }
}

__device__ __forceinline__ void df_add(float &hi, float &lo, float h2, float l2)
{
    const float s = __fadd_rn(hi, h2);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(l2, err));
}

// y = H_local x and, with kS, S_local x in one pass (both feed the same
// Gram-Schmidt step and share the local block list, so the x gathers and the
// index reads serve both).  Lanes run over local block rows, so the
// local-structure reads coalesce and the x gathers stay inside the columns'
// short local vectors.  FP32: H by exact products and two-sums over its hi + lo
// values, output as a (hi, lo) pair (the subspace matrix entries use it), S by
// FMAs over its hi values; FP64: FMAs.  Rows whose support tile lies more than
// `lim` hops from the column's atom are exact zeros and are written without
// being computed.
//
// The NC batch columns c0 .. c0 + NC - 1 belong to one atom here: a column's
// region, local block lists and tile order depend only on its atom, so one
// pass over the blocks, each block read once, serves all NC columns (the
// lanes read different blocks, so the block reads are what the L1 spends its
// time on).  Every column's sums run in the same order as alone.
template <typename VT, bool kS, int NC>
__device__ __forceinline__ void regional_rows(
    int p, int c0, int n_reg, int maxrow, const int *__restrict__ lcnt, const int *__restrict__ lci,
    const int *__restrict__ lgk, const VT *__restrict__ Hv, const VT *__restrict__ Sv,
    const VT *__restrict__ X, int64_t ldx, VT *__restrict__ U, VT *__restrict__ Ulo, int64_t ldu,
    VT *__restrict__ SY, int64_t ldsy, int ncols, const uint8_t *__restrict__ thop,
    const uint16_t *__restrict__ tinv, int lim)
{
    constexpr bool kF = sizeof(VT) == 4;
    constexpr int stride = kF ? 32 : 16;
    const int64_t base = (int64_t)c0 * maxrow * n_reg;
    const bool act = (int)thop[(int64_t)(p >> 3) * ncols + c0] <= lim;
    const int cnt = act ? lcnt[(int64_t)c0 * n_reg + p] : 0;
    VT acc[NC][4], acl[NC][4], sacc[NC][4];
#pragma unroll
    for (int m = 0; m < NC; ++m)
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[m][a] = acl[m][a] = sacc[m][a] = VT(0);
    for (int s = 0; s < cnt; ++s) {
        const int q = lci[base + (int64_t)s * n_reg + p];
        const int64_t k = lgk[base + (int64_t)s * n_reg + p];
        if (!in_range(q, n_reg, kChkRegionCol)) continue;
        const int64_t xp = 32 * (int64_t)tinv[(int64_t)(q >> 3) * ncols + c0] + 4 * (q & 7);
        if (!in_range(xp, ldu - 3, kChkRegionGather)) continue;
        VT xv[NC][4];
#pragma unroll
        for (int m = 0; m < NC; ++m) load4(X + (int64_t)(c0 + m) * ldx + xp, xv[m]);
        const VT *Hb = Hv + stride * k;
        const VT *Sb = Sv + stride * k;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            VT hr[4], lr[4], sr[4];
            load4(Hb + 4 * a, hr);
            if constexpr (kF) load4(Hb + 16 + 4 * a, lr);
            if constexpr (kS) load4(Sb + 4 * a, sr);
#pragma unroll
            for (int m = 0; m < NC; ++m) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if constexpr (kF) {
                        const float pr = __fmul_rn(hr[e], xv[m][e]);
                        const float er = __fmaf_rn(hr[e], xv[m][e], -pr);
                        df_add(acc[m][a], acl[m][a], pr, __fmaf_rn(lr[e], xv[m][e], er));
                    } else {
                        acc[m][a] = fma(hr[e], xv[m][e], acc[m][a]);
                    }
                    if constexpr (kS) sacc[m][a] = fma(sr[e], xv[m][e], sacc[m][a]);
                }
            }
        }
    }
    const int64_t yp = 32 * (int64_t)tinv[(int64_t)(p >> 3) * ncols + c0] + 4 * (p & 7);
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const int64_t c = c0 + m;
        if constexpr (kF) {
            VT yh[4], yl[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                yh[a] = __fadd_rn(acc[m][a], acl[m][a]);
                yl[a] = __fsub_rn(acl[m][a], __fsub_rn(yh[a], acc[m][a]));
            }
            store4(U + c * ldu + yp, yh);
            store4(Ulo + c * ldu + yp, yl);
        } else {
            store4(U + c * ldu + yp, acc[m]);
        }
        if constexpr (kS) store4(SY + c * ldsy + yp, sacc[m]);
    }
}

// Thread (x, y) of a 32x8 CTA: local row p = 32 blockIdx.x + x of group
// g = 8 blockIdx.y + y, the batch columns gstart[g] .. gstart[g + 1] - 1 of one
// atom (the host splits the batch into runs of one atom's columns of at most
// G = reg_group<VT>()).  A full group takes one shared pass; a shorter one (an
// atom with fewer real orbitals, or a run cut by the batch) runs its columns
// one by one.  G is what the registers allow: FP64 accumulators for four
// columns would leave one CTA per SM.
template <typename VT>
constexpr int reg_group()
{
    return sizeof(VT) == 4 ? 4 : 2;
}

template <typename VT, bool kS>
__global__ void __launch_bounds__(256) spmm_regional_hs_kernel(
    int n_reg, int maxrow, const int *__restrict__ lcnt, const int *__restrict__ lci,
    const int *__restrict__ lgk, const VT *__restrict__ Hv, const VT *__restrict__ Sv,
    const VT *__restrict__ X, int64_t ldx, VT *__restrict__ U, VT *__restrict__ Ulo, int64_t ldu,
    VT *__restrict__ SY, int64_t ldsy, int ncols, const int *__restrict__ gstart, int ngroups,
    const uint8_t *__restrict__ thop, const uint16_t *__restrict__ tinv, int lim)
{
    constexpr int G = reg_group<VT>();
    const int p = blockIdx.x * 32 + threadIdx.x;
    const int g = blockIdx.y * 8 + threadIdx.y;
    if (p >= n_reg || g >= ngroups) return;
    // clipped to ncols: a run of the autotuner covers the batch's first columns only
    const int c0 = gstart[g], c1 = min(gstart[g + 1], ncols);
    if (c0 >= c1) return;
    if (c1 - c0 == G) {
        regional_rows<VT, kS, G>(p, c0, n_reg, maxrow, lcnt, lci, lgk, Hv, Sv, X, ldx, U, Ulo, ldu, SY, ldsy,
                                 ncols, thop, tinv, lim);
    } else {
#pragma unroll 1
        for (int c = c0; c < c1; ++c)
            regional_rows<VT, kS, 1>(p, c, n_reg, maxrow, lcnt, lci, lgk, Hv, Sv, X, ldx, U, Ulo, ldu, SY, ldsy,
                                     ncols, thop, tinv, lim);
    }
}

}  // namespace

int regional_group(int prec) { return prec == 0 ? reg_group<double>() : reg_group<float>(); }

cudaError_t launch_spmm_regional_hs(const DeviceMatrix &A, const RegionMaps &rm, const KrylovBatch &b,
                                    const void *X, int64_t ldx, void *SY, int64_t ldsy, int lim,
                                    cudaStream_t s)
{
    if (!b.thop || !b.tinv || b.ntile * 8 < rm.n_reg) return cudaErrorInvalidValue;
    const dim3 block(32, 8);
    if (!rm.gstart || rm.ngroups < 1) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((rm.n_reg + 31) / 32), (unsigned)((rm.ngroups + 7) / 8));
    const int64_t ldu = b.shape.m_pad;
    if (b.prec == 0) {
        if (SY)
            spmm_regional_hs_kernel<double, true><<<grid, block, 0, s>>>(
                rm.n_reg, rm.maxrow, rm.lcnt, rm.lci, rm.lgk, A.Hd, A.Sd, (const double *)X, ldx, (double *)b.U,
                nullptr, ldu, (double *)SY, ldsy, b.nb, rm.gstart, rm.ngroups, b.thop, b.tinv, lim);
        else
            spmm_regional_hs_kernel<double, false><<<grid, block, 0, s>>>(
                rm.n_reg, rm.maxrow, rm.lcnt, rm.lci, rm.lgk, A.Hd, A.Sd, (const double *)X, ldx, (double *)b.U,
                nullptr, ldu, nullptr, 0, b.nb, rm.gstart, rm.ngroups, b.thop, b.tinv, lim);
    } else {
        if (SY)
            spmm_regional_hs_kernel<float, true><<<grid, block, 0, s>>>(
                rm.n_reg, rm.maxrow, rm.lcnt, rm.lci, rm.lgk, A.Hf, A.Sf, (const float *)X, ldx, (float *)b.U,
                (float *)b.Ulo, ldu, (float *)SY, ldsy, b.nb, rm.gstart, rm.ngroups, b.thop, b.tinv, lim);
        else
            spmm_regional_hs_kernel<float, false><<<grid, block, 0, s>>>(
                rm.n_reg, rm.maxrow, rm.lcnt, rm.lci, rm.lgk, A.Hf, A.Sf, (const float *)X, ldx, (float *)b.U,
                (float *)b.Ulo, ldu, nullptr, 0, b.nb, rm.gstart, rm.ngroups, b.thop, b.tinv, lim);
    }
    return cudaGetLastError();
}

cudaError_t launch_region(const RegionMaps &rm, const KrylovBatch &b, double rs, int cap,
                          cudaStream_t s)
{
    const int hx = (int)ceil(rs / rm.cell_edge[0]), hy = (int)ceil(rs / rm.cell_edge[1]),
              hz = (int)ceil(rs / rm.cell_edge[2]);
    const size_t smem = (size_t)cap * (sizeof(double) + sizeof(int));
    cudaError_t e = allow_dynamic_smem((const void *)region_kernel, smem);
    if (e != cudaSuccess) return e;
    region_kernel<<<b.nb, 1024, smem, s>>>(rm.pos, rm.box, rm.cell_start, rm.cell_atoms,
                                           make_int3(rm.ncell[0], rm.ncell[1], rm.ncell[2]),
                                           rm.cell_edge[0], rm.cell_edge[1], rm.cell_edge[2],
                                           b.cols, rm.n_reg, rs * rs, hx, hy, hz, cap, rm.reg,
                                           rm.rstat);
    return cudaGetLastError();
}

cudaError_t launch_local_bsr(const DeviceMatrix &A, const RegionMaps &rm, const KrylovBatch &b,
                             cudaStream_t s)
{
    const dim3 grid((unsigned)((rm.n_reg + 255) / 256), (unsigned)b.nb);
    local_bsr_kernel<<<grid, 256, 0, s>>>(A.rp, A.ci, b.cols, rm.reg, rm.n_reg, rm.maxrow, rm.lcnt,
                                          rm.lci, rm.lgk);
    return cudaGetLastError();
}

cudaError_t launch_init_regional(const DeviceMatrix &A, const RegionMaps &rm, const KrylovBatch &b,
                                 cudaStream_t s)
{
    if (b.prec == 0)
        init_regional_kernel<double><<<b.nb, 256, 0, s>>>(
            A.Sd, A.sdiag, b.cols, rm.reg, rm.n_reg, rm.maxrow, rm.lcnt, rm.lci, rm.lgk,
            (double *)b.K, (double *)b.SK, b.scale, b.status, b.nu_eff, b.nu, b.shape.m_pad,
            b.tinv, b.nb);
    else
        init_regional_kernel<float><<<b.nb, 256, 0, s>>>(
            A.Sd, A.sdiag, b.cols, rm.reg, rm.n_reg, rm.maxrow, rm.lcnt, rm.lci, rm.lgk,
            (float *)b.K, (float *)b.SK, b.scale, b.status, b.nu_eff, b.nu, b.shape.m_pad,
            b.tinv, b.nb);
    return cudaGetLastError();
}


MARNOLDI_CHECK_TAKE(region)

}  // namespace marnoldi
