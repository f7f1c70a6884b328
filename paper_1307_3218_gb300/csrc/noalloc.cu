// Electron count and band energy over subspace levels without allocating.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory manager with a fixed budget, or a service that must not
// allocate on its request path.  marnoldi_count_noalloc gives them the
// electron-count reduction (the per-step work of the Fermi-level bisection)
// with its scratch in a fixed device array that the library owns: the
// per-block partial sums and the completion ticket live in g_count_scratch,
// a file-scope __device__ array of 64 KiB + 16 bytes that every GPU which
// loads the library keeps until the process exits.
//
// Each block reduces one fixed chunk of kChunk levels, so the scratch bounds
// the input: at most kMaxBlocks * kChunk = 16,777,216 levels per call.
#include "marnoldi.h"
#include "internal.h"

#include <cuda_runtime.h>

#include <cmath>

namespace marnoldi {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 4096;                       // levels per block
constexpr int kMaxBlocks = 4096;                   // partial-sum slots
constexpr int64_t kMaxLevels = (int64_t)kChunk * kMaxBlocks;
static_assert(kMaxLevels == MARNOLDI_COUNT_NOALLOC_MAX_LEVELS, "the header states the limit");
constexpr int kScratchDoubles = 2 * kMaxBlocks + 2; // partials, then the ticket

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) double g_count_scratch[kScratchDoubles];

// The device address of g_count_scratch is looked up on every call (host
// code cannot use the symbol itself: on the host it names a stand-in, not
// device memory).  The lookup allocates nothing, and a cached address would
// go stale if the device's primary context were reset and the module loaded
// again at another address.

__device__ __forceinline__ double fermi_na(double x)
{
    if (x >= 0.0) {
        const double e = exp(-x);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + exp(x));
}

__global__ void __launch_bounds__(kThreads) count_noalloc_kernel(
    int64_t total, int nu, const int32_t *__restrict__ nu_eff, const double *__restrict__ eps,
    const double *__restrict__ w, double mu, double kT, double *scratch, double *out)
{
    __shared__ double2 red[kThreads / 32];
    __shared__ int last;
    const int64_t b0 = (int64_t)blockIdx.x * kChunk;
    const int64_t b1 = b0 + kChunk < total ? b0 + kChunk : total;
    double sn = 0.0, se = 0.0;
    for (int64_t idx = b0 + threadIdx.x; idx < b1; idx += kThreads) {
        const int64_t c = idx / nu;
        if (nu_eff == nullptr || idx - c * nu < nu_eff[c]) {
            const double ea = eps[idx];
            const double f2w = 2.0 * fermi_na((ea - mu) / kT) * w[idx];
            sn += f2w;
            se = fma(f2w, ea, se);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sn += __shfl_xor_sync(0xffffffffu, sn, o);
        se += __shfl_xor_sync(0xffffffffu, se, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double2(sn, se);
    __syncthreads();
    unsigned *ticket = reinterpret_cast<unsigned *>(scratch + 2 * kMaxBlocks);
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) {
            x += red[q].x;
            y += red[q].y;
        }
        scratch[2 * blockIdx.x] = x;
        scratch[2 * blockIdx.x + 1] = y;
        __threadfence();
        last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const volatile double *vp = scratch;
        double x = 0.0, y = 0.0;
        for (unsigned q = 0; q < gridDim.x; ++q) {
            x += vp[2 * q];
            y += vp[2 * q + 1];
        }
        out[0] = x;
        out[1] = y;
        *ticket = 0u;
    }
}

// Set-up, on every call with the caller's device current: the device address
// of the scratch array on that device.  Returns nullptr on failure.
double *scratch_for_current_device(cudaError_t *err)
{
    double *p = nullptr;
    *err = cudaGetSymbolAddress((void **)&p, g_count_scratch);
    return *err == cudaSuccess ? p : nullptr;
}

}  // namespace
}  // namespace marnoldi

extern "C" int marnoldi_count_noalloc(const double *eps_device, const double *w_device,
                                      const int32_t *nu_eff_device, int64_t ncols, int nu,
                                      double mu, double kT, double *out_device, void *cuda_stream)
{
    using namespace marnoldi;
    if (!eps_device || !w_device || !out_device)
        return set_global_error(MARNOLDI_EINVAL, "count_noalloc: NULL device pointer");
    if (ncols < 1 || nu < 1)
        return set_global_error(MARNOLDI_EINVAL, "count_noalloc: ncols and nu must be >= 1");
    if (!(kT > 0.0) || !std::isfinite(kT) || !std::isfinite(mu))
        return set_global_error(MARNOLDI_EINVAL, "count_noalloc: kT must be positive, mu finite");
    if (ncols > kMaxLevels / nu)
        return set_global_error(MARNOLDI_EINVAL,
                                "count_noalloc: ncols * nu exceeds the maximum of 16777216 levels "
                                "of the fixed scratch; split the levels over several calls");
    const int64_t total = ncols * (int64_t)nu;
    cudaError_t e = cudaSuccess;
    double *scratch = scratch_for_current_device(&e);
    if (!scratch) return set_global_error(MARNOLDI_ECUDA, "count_noalloc: scratch set-up failed");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the ticket must start at zero (a memset, not an allocation)
    e = cudaMemsetAsync(scratch + 2 * kMaxBlocks, 0, sizeof(double), s);
    if (e != cudaSuccess) return set_global_error(MARNOLDI_ECUDA, "count_noalloc: ticket clear failed");
    const unsigned blocks = (unsigned)((total + kChunk - 1) / kChunk);
    count_noalloc_kernel<<<blocks, kThreads, 0, s>>>(total, nu, nu_eff_device, eps_device, w_device,
                                                     mu, kT, scratch, out_device);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_global_error(MARNOLDI_ECUDA, "count_noalloc: launch failed");
    return MARNOLDI_OK;
}
