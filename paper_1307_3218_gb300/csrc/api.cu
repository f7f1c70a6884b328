// Host side of libmarnoldi: the exported C ABI (include/marnoldi.h), input
// validation, device memory, the batch loop over columns, and the Fermi-level
// bisection (one device reduction and one 16-byte read-back per step).
#include "marnoldi.h"
#include "internal.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <iterator>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>
#include <utility>
#include <vector>

using namespace marnoldi;

namespace {

marnoldi_alloc_fn g_alloc = nullptr;
marnoldi_free_fn g_free = nullptr;
void *g_user = nullptr;
thread_local std::string g_setup_err;

constexpr double kTauFp64 = 1e-10;
constexpr double kTauMixed = 1e-5;

// Reduction scratch of a context: partial sums, the reduction output, the
// level range, the bisection state and the reductions' ticket.
constexpr size_t kOffOut = 2 * kReduceBlocks * sizeof(double);
constexpr size_t kOffRange = kOffOut + 2 * sizeof(double);
constexpr size_t kOffBisect = kOffRange + 2 * sizeof(double);
constexpr size_t kOffTicket = kOffBisect + ((sizeof(BisectState) + 15) & ~(size_t)15);
constexpr size_t kScratchBytes = kOffTicket + 16;

}  // namespace

int marnoldi::set_global_error(int code, const char *msg)
{
    g_setup_err = msg;
    return code;
}

cudaError_t marnoldi::allow_dynamic_smem(const void *kernel, size_t bytes)
{
    static std::mutex mu;
    static std::unordered_map<const void *, size_t> allowed;
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = allowed[kernel];
    if (bytes <= cur) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

namespace {

// Page-locked read-back slots of 128 bytes, carved from pages that stay
// allocated until the process exits, so that creating and destroying a
// context never calls cudaMallocHost or cudaFreeHost (either may wait for
// work that other streams have in flight).
std::mutex g_pin_mu;
std::vector<double *> g_pin_free;

double *pinned_slot()
{
    std::lock_guard<std::mutex> lock(g_pin_mu);
    if (g_pin_free.empty()) {
        void *page = nullptr;
        if (cudaMallocHost(&page, 4096) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (int q = 0; q < 4096 / 128; ++q) g_pin_free.push_back((double *)page + 16 * q);
    }
    double *slot = g_pin_free.back();
    g_pin_free.pop_back();
    return slot;
}

void pinned_release(double *slot)
{
    if (!slot) return;
    std::lock_guard<std::mutex> lock(g_pin_mu);
    g_pin_free.push_back(slot);
}

}  // namespace

namespace {

// ---- autotuner of the Gram-Schmidt launch shape.  Shapes with the same
// m_pad differ in threads per CTA and values per thread; the choice changes
// the order of the kernel's partial sums (so results by rounding) and its
// speed.  Mode 0 (default): the fixed rule of column_shape.  Mode 1: the first
// solve of a (precision, nu, mode, m_pad) key times every candidate on its
// first kTuneColumns columns and keeps the fastest for the process; with
// MARNOLDI_TUNE_CACHE=<file> the choices are read from and appended to that
// file, so later processes reuse them.
constexpr int64_t kTuneColumns = 1216;   // 8 CTAs per SM on 152 SMs

struct TuneKey {
    int prec, nu, regional;
    int64_t m_pad;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(prec, nu, regional, m_pad) < std::tie(o.prec, o.nu, o.regional, o.m_pad);
    }
};

std::mutex g_tune_mu;
std::map<TuneKey, ColumnShape> g_tuned;
int g_autotune = -1;   // -1: not read from MARNOLDI_AUTOTUNE yet
bool g_tune_cache_loaded = false;

int autotune_mode()
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (g_autotune < 0) {
        const char *v = getenv("MARNOLDI_AUTOTUNE");
        g_autotune = (v && v[0] == '1') ? 1 : 0;
    }
    return g_autotune;
}

void load_tune_cache_locked()
{
    if (g_tune_cache_loaded) return;
    g_tune_cache_loaded = true;
    const char *path = getenv("MARNOLDI_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    TuneKey k;
    long long mp;
    int v, t;
    while (fscanf(f, "%d %d %d %lld %d %d", &k.prec, &k.nu, &k.regional, &mp, &v, &t) == 6) {
        k.m_pad = mp;
        ColumnShape cand[kMaxShapes];
        const int n = column_shape_candidates(k.m_pad, k.prec, cand);
        for (int q = 0; q < n; ++q)   // only shapes the library is compiled for
            if (cand[q].vpt == v && cand[q].threads == t) g_tuned[k] = cand[q];
    }
    fclose(f);
}

void save_tune_entry_locked(const TuneKey &k, const ColumnShape &s)
{
    const char *path = getenv("MARNOLDI_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%d %d %d %lld %d %d\n", k.prec, k.nu, k.regional, (long long)k.m_pad, s.vpt, s.threads);
    fclose(f);
}

}  // namespace

struct marnoldi_ctx {
    cudaStream_t stream = nullptr;
    int prec = 0;
    int64_t nbr = 0, nnzb = 0, m = 0;
    int maxrow = 1;   // most blocks in a block row
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<uint8_t> mask;
    std::vector<double> pos, box;
    marnoldi_alloc_fn alloc = nullptr;
    marnoldi_free_fn free_fn = nullptr;
    void *user = nullptr;

    // device memory: bytes held now and at most since setup
    size_t dev_bytes = 0, dev_peak = 0;

    // device copies of the structure
    DeviceMatrix A{};
    std::vector<std::pair<void *, size_t>> owned;  // structure + scratch allocations

    // reduction scratch and pinned read-back
    double *d_partial = nullptr;
    unsigned *d_ticket = nullptr;
    double *d_out = nullptr, *d_range = nullptr;
    BisectState *d_bisect = nullptr;
    double *h_out = nullptr;   // 128-byte pinned read-back slot

    // solved state
    bool solved = false;
    int64_t ncols = 0;
    int nu = 0;
    double mu = 0.0, N = 0.0, E = 0.0, kT = 0.0;
    std::vector<int64_t> cols;
    void *state = nullptr;
    size_t state_bytes = 0;
    ColumnState st{};
    int64_t *d_cols = nullptr;

    // batch workspace
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int64_t batch_override = 0;
    int64_t last_batch = 0;
    ColumnShape gs_shape{0, 0, 0};   // Gram-Schmidt launch shape of the last solve
    KrylovBatch last_kb{};           // the last batch of the last solve (its workspace stays)
    bool last_regional = false, last_all_real = false;
    // projection of the stored vectors on proj_vec (M rows, device), turned
    // by the eigensolve into proj_out[g * nu + a] = proj_vec^T K v_a
    const double *proj_vec = nullptr;
    double *proj_out = nullptr;
    bool shares_structure = false;   // a view of another context's device structure

    // members: a block-diagonal union of independent structures (atom ranges
    // starting at multiples of 8 atoms), each with its own electron count and
    // Fermi level, solved in the same launches
    std::vector<int64_t> mem_atom;   // n + 1 atom offsets (empty: one structure)
    std::vector<double> mem_ne;
    std::vector<double> mem_kT;   // per-member kT (empty: the solve's kT for every member)
    std::vector<int64_t> mem_col;    // n + 1 offsets into the solved columns
    std::vector<double> mem_mu, mem_N, mem_E;

    // regional mode: positions, box, cell list (built on first use) and the
    // last search radius that worked
    bool cells_ready = false;
    RegionMaps rm{};
    double region_rs = 0.0;

    // the Krylov build of a batch as one CUDA graph (marnoldi_set_krylov_graph):
    // captured from the stream on every batch, the executable graph kept and
    // updated in place while the topology (nu, mode) stays the same
    bool krylov_graph = false;
    cudaGraphExec_t kexec = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream the graph is captured from
    int64_t graph_launches = 0;

    // instrumentation
    int64_t launches[KK_NKINDS] = {};
    double ms[KK_NKINDS] = {};
    int profile = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    std::vector<cudaEvent_t> events;

    std::string err;
};

namespace {

int fail(marnoldi_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_setup_err = buf;
    return code;
}

int fail_cuda(marnoldi_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, MARNOLDI_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *dalloc(marnoldi_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (c->alloc) {
        p = c->alloc(bytes, (void *)c->stream, c->user);
    } else if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        c->dev_bytes += bytes;
        c->dev_peak = std::max(c->dev_peak, c->dev_bytes);
    }
    return p;
}

void dfree(marnoldi_ctx *c, void *p, size_t bytes)
{
    if (!p) return;
    if (bytes == 0) bytes = 16;
    c->dev_bytes -= bytes;
    if (c->free_fn) c->free_fn(p, bytes, (void *)c->stream, c->user);
    else cudaFreeAsync(p, c->stream);
}

// A device allocation of a context released (in stream order) at scope exit.
struct DeviceBuffer {
    marnoldi_ctx *c;
    size_t bytes;
    double *p;
    DeviceBuffer(marnoldi_ctx *ctx, size_t n) : c(ctx), bytes(n), p(n ? (double *)dalloc(ctx, n) : nullptr) {}
    ~DeviceBuffer() { if (p) dfree(c, p, bytes); }
    DeviceBuffer(const DeviceBuffer &) = delete;
    DeviceBuffer &operator=(const DeviceBuffer &) = delete;
    double *get() const { return p; }
};

template <typename T>
int dupload(marnoldi_ctx *c, T **dst, const T *src, size_t n, const char *what)
{
    const size_t bytes = n * sizeof(T);
    void *p = dalloc(c, bytes);
    if (!p) return fail(c, MARNOLDI_ENOMEM, "device allocation of %zu bytes for %s failed", bytes, what);
    c->owned.push_back({p, bytes});
    *dst = (T *)p;
    if (n) {
        cudaError_t e = cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return fail_cuda(c, e, what);
    }
    return MARNOLDI_OK;
}

cudaEvent_t get_event(marnoldi_ctx *c)
{
    if (!c->events.empty()) {
        cudaEvent_t e = c->events.back();
        c->events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// NVTX range over one phase of a call (host timeline: when its launches are
// issued and, for the phases that end in a synchronisation, until they end).
// A profiler shows them; without one the calls cost next to nothing.
struct Phase {
    explicit Phase(const char *name) { nvtxRangePushA(name); }
    ~Phase() { nvtxRangePop(); }
    Phase(const Phase &) = delete;
    Phase &operator=(const Phase &) = delete;
};

void collect_profile(marnoldi_ctx *c)
{
    for (auto &p : c->pending) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p.second.first, p.second.second) == cudaSuccess)
            c->ms[p.first] += t;
        c->events.push_back(p.second.first);
        c->events.push_back(p.second.second);
    }
    c->pending.clear();
    cudaGetLastError();
}

template <typename F>
int launch(marnoldi_ctx *c, int kind, F &&f)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profile) {
        e0 = get_event(c);
        e1 = get_event(c);
        cudaEventRecord(e0, c->stream);
    }
    cudaError_t e = f();
    if (e != cudaSuccess) return fail_cuda(c, e, kernel_name(kind));
    if (c->profile) {
        cudaEventRecord(e1, c->stream);
        c->pending.push_back({kind, {e0, e1}});
    }
    c->launches[kind]++;
    return MARNOLDI_OK;
}

// Run `body` (stream work on c->stream only) as one CUDA graph: capture it
// from a private stream of the context (the context's own stream may be the
// legacy default stream, which cannot be captured), update the kept
// executable graph in place (or instantiate one when the topology changed)
// and launch it on the context's stream, after the work already queued there.
// A failed launch inside the body ends the capture and returns the body's
// error.
template <class F>
int run_as_graph(marnoldi_ctx *c, F &&body)
{
    cudaError_t e;
    if (!c->cap_stream && (e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        c->cap_stream = nullptr;
        return fail_cuda(c, e, "Krylov graph stream");
    }
    if ((e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return fail_cuda(c, e, "Krylov graph capture");
    const cudaStream_t own = c->stream;
    c->stream = c->cap_stream;
    const int r = body();
    c->stream = own;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &g);
    if (r || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return r ? r : fail_cuda(c, e, "Krylov graph capture");
    }
    bool updated = false;
    if (c->kexec) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(c->kexec, g, &info) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();
            cudaGraphExecDestroy(c->kexec);
            c->kexec = nullptr;
        }
    }
    if (!updated && (e = cudaGraphInstantiate(&c->kexec, g, 0)) != cudaSuccess) {
        c->kexec = nullptr;
        cudaGraphDestroy(g);
        return fail_cuda(c, e, "Krylov graph instantiation");
    }
    cudaGraphDestroy(g);
    if ((e = cudaGraphLaunch(c->kexec, c->stream)) != cudaSuccess) return fail_cuda(c, e, "Krylov graph launch");
    c->graph_launches++;
    return MARNOLDI_OK;
}

int sync(marnoldi_ctx *c, const char *what)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e, what);
    if (c->profile) collect_profile(c);
    return MARNOLDI_OK;
}

// Smallest eigenvalue of a symmetric tridiagonal matrix (diag a, off b) by
// Sturm-sequence bisection.
double tridiag_min_eig(const std::vector<double> &a, const std::vector<double> &b)
{
    const int n = (int)a.size();
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    for (int it = 0; it < 200; ++it) {
        const double x = 0.5 * (lo + hi);
        int neg = 0;
        double q = 1.0;
        for (int i = 0; i < n; ++i) {
            q = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0.0) ++neg;
        }
        if (neg >= 1) hi = x; else lo = x;
        if (hi - lo <= 1e-14 * std::max(1.0, std::fabs(hi))) break;
    }
    return lo;
}

// Lowest Ritz value of S after `steps` plain Lanczos steps from a fixed
// pseudo-random start on the real orbitals.  Ritz values lie inside S's
// spectrum, so a value <= 0 proves S is not positive definite.
double lanczos_min_ritz(const marnoldi_ctx *c, const double *Sv, int steps)
{
    const int64_t M = c->m;
    std::vector<double> v(M, 0.0), vp(M, 0.0), wv(M, 0.0);
    uint64_t st = 0x9E3779B97F4A7C15ull;
    double nrm = 0.0;
    for (int64_t r = 0; r < M; ++r) {
        st ^= st << 13; st ^= st >> 7; st ^= st << 17;
        const double x = c->mask.empty() || c->mask[r] ? ((double)(st >> 11) / 9007199254740992.0 - 0.5) : 0.0;
        v[r] = x;
        nrm += x * x;
    }
    nrm = std::sqrt(nrm);
    for (auto &x : v) x /= nrm;
    std::vector<double> a, b;
    double beta = 0.0;
    for (int s = 0; s < steps; ++s) {
        for (int64_t I = 0; I < c->nbr; ++I) {
            double acc[4] = {0, 0, 0, 0};
            for (int64_t k = c->rp[I]; k < c->rp[I + 1]; ++k) {
                const double *B = Sv + 16 * k;
                const double *x = v.data() + 4 * (int64_t)c->ci[k];
                for (int p = 0; p < 4; ++p)
                    for (int q = 0; q < 4; ++q) acc[p] += B[4 * p + q] * x[q];
            }
            for (int p = 0; p < 4; ++p) wv[4 * I + p] = acc[p];
        }
        double alpha = 0.0;
        for (int64_t r = 0; r < M; ++r) alpha += wv[r] * v[r];
        for (int64_t r = 0; r < M; ++r) wv[r] -= alpha * v[r] + beta * vp[r];
        a.push_back(alpha);
        double nb = 0.0;
        for (int64_t r = 0; r < M; ++r) nb += wv[r] * wv[r];
        nb = std::sqrt(nb);
        if (!(nb > 1e-12) || s + 1 == steps) break;
        b.push_back(nb);
        beta = nb;
        vp.swap(v);
        for (int64_t r = 0; r < M; ++r) v[r] = wv[r] / nb;
    }
    b.resize(a.size() > 0 ? a.size() - 1 : 0);
    return tridiag_min_eig(a, b);
}

int validate_structure(marnoldi_ctx *c, const double *H, const double *S)
{
    const int64_t nbr = c->nbr;
    const auto &rp = c->rp;
    const auto &ci = c->ci;
    if (rp[0] != 0) return fail(nullptr, MARNOLDI_EINVAL, "row_ptr[0] must be 0");
    for (int64_t I = 0; I < nbr; ++I) {
        if (rp[I + 1] < rp[I]) return fail(nullptr, MARNOLDI_EINVAL, "row_ptr decreases at %lld", (long long)I);
        bool diag = false;
        for (int64_t k = rp[I]; k < rp[I + 1]; ++k) {
            if (ci[k] < 0 || ci[k] >= nbr)
                return fail(nullptr, MARNOLDI_EINVAL, "col_idx[%lld] = %d out of range", (long long)k, ci[k]);
            if (k > rp[I] && ci[k] <= ci[k - 1])
                return fail(nullptr, MARNOLDI_EINVAL, "col_idx not strictly ascending in block row %lld", (long long)I);
            if (ci[k] == I) diag = true;
        }
        if (!diag) return fail(nullptr, MARNOLDI_EINVAL, "block row %lld has no diagonal block", (long long)I);
    }
    // symmetry of pattern and values
    double hmax = 0.0, smax = 0.0;
    for (int64_t k = 0; k < 16 * c->nnzb; ++k) {
        if (!std::isfinite(H[k]) || !std::isfinite(S[k]))
            return fail(nullptr, MARNOLDI_EINVAL, "non-finite matrix value in block %lld", (long long)(k / 16));
        hmax = std::max(hmax, std::fabs(H[k]));
        smax = std::max(smax, std::fabs(S[k]));
    }
    for (int64_t I = 0; I < nbr; ++I) {
        for (int64_t k = rp[I]; k < rp[I + 1]; ++k) {
            const int64_t J = ci[k];
            const int32_t *b0 = ci.data() + rp[J], *b1 = ci.data() + rp[J + 1];
            const int32_t *f = std::lower_bound(b0, b1, (int32_t)I);
            if (f == b1 || *f != (int32_t)I)
                return fail(nullptr, MARNOLDI_EINVAL, "pattern not symmetric: block (%lld,%lld) has no mirror",
                            (long long)I, (long long)J);
            const int64_t kt = rp[J] + (f - b0);
            for (int a = 0; a < 4; ++a)
                for (int bb = 0; bb < 4; ++bb) {
                    if (std::fabs(H[16 * k + 4 * a + bb] - H[16 * kt + 4 * bb + a]) > 1e-12 * hmax)
                        return fail(nullptr, MARNOLDI_EINVAL, "H not symmetric in block (%lld,%lld)", (long long)I, (long long)J);
                    if (std::fabs(S[16 * k + 4 * a + bb] - S[16 * kt + 4 * bb + a]) > 1e-12 * smax)
                        return fail(nullptr, MARNOLDI_EINVAL, "S not symmetric in block (%lld,%lld)", (long long)I, (long long)J);
                    if (!c->mask.empty() && c->mask[4 * I + a] != c->mask[4 * J + bb] &&
                        (H[16 * k + 4 * a + bb] != 0.0 || S[16 * k + 4 * a + bb] != 0.0))
                        return fail(nullptr, MARNOLDI_EINVAL, "padding orbital couples to a real orbital in block (%lld,%lld)",
                                    (long long)I, (long long)J);
                }
        }
    }
    // S_jj > 0 for real orbitals; Lanczos lower Ritz value
    for (int64_t I = 0; I < nbr; ++I)
        for (int64_t k = rp[I]; k < rp[I + 1]; ++k)
            if (ci[k] == I)
                for (int a = 0; a < 4; ++a)
                    if ((c->mask.empty() || c->mask[4 * I + a]) && !(S[16 * k + 5 * a] > 0.0))
                        return fail(nullptr, MARNOLDI_ENOTSPD, "S_jj <= 0 at orbital %lld", (long long)(4 * I + a));
    const double ritz = lanczos_min_ritz(c, S, 40);
    if (!(ritz > 0.0))
        return fail(nullptr, MARNOLDI_ENOTSPD, "S is not positive definite (Lanczos Ritz value %.3e)", ritz);
    return MARNOLDI_OK;
}

// Regional mode, once per context: positions wrapped into the box, a cell list
// of edge >= 2.6 A (counting sort of atoms by cell), and the longest block row.
int build_cells(marnoldi_ctx *c)
{
    if (c->cells_ready) return MARNOLDI_OK;
    const int64_t n = c->nbr;
    for (int d = 0; d < 3; ++d)
        if (!(c->box[d] > 0.0) || !std::isfinite(c->box[d]))
            return fail(c, MARNOLDI_EINVAL, "box lengths must be positive and finite");
    std::vector<double> pos(3 * n);
    for (int64_t a = 0; a < n; ++a)
        for (int d = 0; d < 3; ++d) {
            double x = std::fmod(c->pos[3 * a + d], c->box[d]);
            if (x < 0.0) x += c->box[d];
            if (!std::isfinite(x)) return fail(c, MARNOLDI_EINVAL, "non-finite atom position");
            pos[3 * a + d] = x;
        }
    RegionMaps &rm = c->rm;
    for (int d = 0; d < 3; ++d) {
        rm.ncell[d] = (int)std::max(1.0, std::min(256.0, std::floor(c->box[d] / 2.6)));
        rm.cell_edge[d] = c->box[d] / rm.ncell[d];
    }
    const int64_t ncells = (int64_t)rm.ncell[0] * rm.ncell[1] * rm.ncell[2];
    std::vector<int> cell_of(n), start(ncells + 1, 0), atoms(n);
    for (int64_t a = 0; a < n; ++a) {
        int ix[3];
        for (int d = 0; d < 3; ++d)
            ix[d] = std::min(rm.ncell[d] - 1, std::max(0, (int)(pos[3 * a + d] / rm.cell_edge[d])));
        cell_of[a] = (ix[2] * rm.ncell[1] + ix[1]) * rm.ncell[0] + ix[0];
        ++start[cell_of[a] + 1];
    }
    for (int64_t q = 0; q < ncells; ++q) start[q + 1] += start[q];
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (int64_t a = 0; a < n; ++a) atoms[fill[cell_of[a]]++] = (int)a;
    rm.maxrow = c->maxrow;
    double *dpos = nullptr, *dbox = nullptr;
    int *dst = nullptr, *dat = nullptr;
    int rc;
    if ((rc = dupload(c, &dpos, pos.data(), pos.size(), "positions")) ||
        (rc = dupload(c, &dbox, c->box.data(), 3, "box")) ||
        (rc = dupload(c, &dst, start.data(), start.size(), "cell starts")) ||
        (rc = dupload(c, &dat, atoms.data(), atoms.size(), "cell atoms")))
        return rc;
    rm.pos = dpos;
    rm.box = dbox;
    rm.cell_start = dst;
    rm.cell_atoms = dat;
    c->cells_ready = true;
    return MARNOLDI_OK;
}

// Regions of a batch: search radius from the mean density (or the last one
// that worked), widened when some region finds fewer than n_reg atoms inside
// it and narrowed when the candidates overflow the kernel's buffer.
int find_regions(marnoldi_ctx *c, const KrylovBatch &kb)
{
    const double vol = c->box[0] * c->box[1] * c->box[2];
    const double rho = (double)c->nbr / vol;
    double rs = c->region_rs;
    if (!(rs > 0.0)) rs = 1.3 * std::cbrt(3.0 * c->rm.n_reg / (4.0 * M_PI * rho)) + 1.0;
    std::vector<int> st(kb.nb);
    for (int attempt = 0; attempt < 16; ++attempt) {
        int rc = launch(c, KK_REGION, [&] { return launch_region(c->rm, kb, rs, kRegionCap, c->stream); });
        if (rc) return rc;
        cudaError_t e = cudaMemcpyAsync(st.data(), c->rm.rstat, (size_t)kb.nb * sizeof(int),
                                        cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return fail_cuda(c, e, "region status read-back");
        if ((rc = sync(c, "region search"))) return rc;
        bool few = false, many = false;
        for (int v : st) {
            few |= v == 1;
            many |= v == 2;
        }
        if (!few && !many) {
            c->region_rs = rs;
            return MARNOLDI_OK;
        }
        if (few && many)
            return fail(c, MARNOLDI_EINVAL, "region search: density too uneven for %d candidates per region",
                        kRegionCap);
        rs *= few ? 1.4 : 0.85;
    }
    return fail(c, MARNOLDI_ENOCONV, "region search radius did not settle");
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device memory of one solve (every piece 256-byte aligned): the per-column
// state, kept until the next solve, and the batch workspace, kept and only
// grown across solves.
struct SolvePlan {
    size_t o_cols, o_poff, o_nue, o_est, o_eps, o_w, o_t, o_P, o_grp, state_bytes;
    int64_t B, ntile;
    ColumnShape shape;
    size_t vs;
    bool a_global;
    EigScratch es;   // sizes and chunk; the caller sets the pointers
    size_t oK, oSK, oU, oUl, oH, oL, oSc, oC, oS, oN, oRg, oRc, oRi, oRk, oRs, oTh, oTo, oTc;
    size_t oED, oEE, oERQ, oERot, oESw, oENs, oEA, ws_bytes;
};

// Workspace bytes per batch column, for the default batch size.
size_t per_column_bytes(const ColumnShape &shape, size_t vs, int nu, int region_atoms, int maxrow)
{
    const size_t reg = region_atoms > 0 ? (size_t)region_atoms * (12 + 8 * (size_t)maxrow) : 0;
    return al256((size_t)2 * nu * shape.m_pad * vs) + (size_t)2 * shape.m_pad * vs +
           (size_t)2 * nu * nu * 8 + (size_t)nu * 8 + 64 + reg + (size_t)(shape.m_pad / 32) * 3 +
           (size_t)(nu + 2) * 4;
}

// Batch size within [1, ncols] and the launch limits (one CTA per column, or
// per column pair).
int64_t clamp_batch(int64_t B, int64_t nc, bool regional)
{
    B = std::min<int64_t>(std::max<int64_t>(B, 1), nc);
    B = std::min<int64_t>(B, regional ? 65535 : 65535 * 32);
    // regional batches hold whole groups of 4 columns, so that the orbitals of
    // one atom, listed together, stay in one batch and share the regional
    // product's block reads
    if (regional && B < nc && B >= 4) B -= B % 4;
    return B;
}

// Offsets and sizes of a solve of nc columns (prow = rows of the columns'
// block patterns, 4 per block) in batches of B (already clamped).  Returns
// false when nu with blocks rows of `maxrow` blocks does not fit the
// eigensolver's shared memory.
bool plan_solve(int64_t m_vec, int prec, int nu, int region_atoms, int maxrow, int64_t nc,
                int64_t prow, int64_t B, int64_t ntile_min, SolvePlan &p)
{
    const bool regional = region_atoms > 0;
    p.o_cols = 0;
    p.o_poff = p.o_cols + al256(nc * 8);
    p.o_nue = p.o_poff + al256(nc * 8);
    p.o_est = p.o_nue + al256(nc * 4);
    p.o_eps = p.o_est + al256(nc * 4);
    p.o_w = p.o_eps + al256((size_t)nc * nu * 8);
    p.o_t = p.o_w + al256((size_t)nc * nu * 8);
    p.o_P = p.o_t + al256((size_t)nc * nu * 8);
    p.o_grp = p.o_P + al256((size_t)prow * nu * 8);
    // regional product groups: at most one per column plus one end mark per batch
    p.state_bytes = p.o_grp + (regional ? al256((size_t)(nc + (nc + B - 1) / B) * 4) : 0);

    p.B = B;
    p.shape = column_shape(m_vec, prec);
    p.vs = prec == 0 ? 8 : 4;
    const size_t mp = (size_t)p.shape.m_pad, vs = p.vs;
    const size_t nt = std::max<size_t>(mp / 32, (size_t)ntile_min);   // 8-atom tiles of the structure
    p.ntile = (int64_t)nt;
    const size_t rg = regional ? (size_t)region_atoms : 0;
    p.oK = 0;
    p.oSK = p.oK + al256((size_t)B * nu * mp * vs);
    p.oU = p.oSK + al256((size_t)B * nu * mp * vs);
    p.oUl = p.oU + al256((size_t)B * mp * vs);
    p.oH = p.oUl + (prec == 1 ? al256((size_t)B * mp * vs) : 0);
    p.oL = p.oH + al256((size_t)B * nu * nu * 8);
    p.oSc = p.oL + al256((size_t)B * nu * nu * 8);
    p.oC = p.oSc + al256((size_t)B * nu * 8);
    p.oS = p.oC + al256((size_t)B * 8);
    p.oN = p.oS + al256((size_t)B * 4);
    p.oRg = p.oN + al256((size_t)B * 4);
    p.oRc = p.oRg + (regional ? al256((size_t)B * rg * 4) : 0);
    p.oRi = p.oRc + (regional ? al256((size_t)B * rg * 4) : 0);
    p.oRk = p.oRi + (regional ? al256((size_t)B * rg * maxrow * 4) : 0);
    p.oRs = p.oRk + (regional ? al256((size_t)B * rg * maxrow * 4) : 0);
    p.oTh = p.oRs + (regional ? al256((size_t)B * 4) : 0);
    p.oTo = p.oTh + al256((size_t)B * nt);
    p.oTc = p.oTo + al256((size_t)B * nt * 2);
    const size_t oEg = p.oTc + al256((size_t)B * (nu + 2) * 4);

    // eigensolve scratch, for chunks of at most es.chunk subspaces; H_sub in
    // shared memory when it fits, else in a global scratch per subspace
    EigScratch &es = p.es;
    es = EigScratch{};
    es.nr_max = 4 * maxrow + 3;   // e_1, q, the pattern rows and an optional projection row
    es.rcap = (int64_t)8 * nu * nu;
    es.scap = (int64_t)40 * nu;
    const size_t kSmemCap = (size_t)227 * 1024;
    p.a_global = eig_smem_bytes(nu, es.nr_max, false) > kSmemCap;
    if (eig_smem_bytes(nu, es.nr_max, p.a_global) > kSmemCap) return false;
    const size_t a_per_sub = p.a_global ? (size_t)nu * (nu | 1) * 8 : 0;
    const size_t per_sub = al256((size_t)(2 + es.nr_max) * nu * 8) + al256((size_t)es.rcap * 16) +
                           al256((size_t)es.scap * 8) + 8 + a_per_sub;
    // the QL kernel runs one subspace per lane and its time hardly grows with the chunk (it is
    // latency-bound), so chunks are as large as 12 GB of scratch allow: at nu = 100 a whole
    // batch of 8,192 columns is one chunk
    es.chunk = (int)std::max<int64_t>(32, std::min<int64_t>(B, (int64_t)(((size_t)12 << 30) / per_sub)));
    const size_t ceig = (size_t)es.chunk;
    p.oED = oEg;
    p.oEE = p.oED + al256(ceig * nu * 8);
    p.oERQ = p.oEE + al256(ceig * nu * 8);
    p.oERot = p.oERQ + al256(ceig * es.nr_max * nu * 8);
    p.oESw = p.oERot + al256(ceig * es.rcap * 16);
    p.oENs = p.oESw + al256(ceig * es.scap * 8);
    p.oEA = p.oENs + al256(ceig * 4);
    p.ws_bytes = p.oEA + al256(ceig * a_per_sub);
    return true;
}

// Device bytes that marnoldi_setup allocates for a structure, and that the
// first regional solve adds (wrapped positions, box, cell list).
size_t setup_bytes(int64_t nbr, int64_t nnzb, int prec)
{
    size_t b = 8 * (size_t)(nbr + 1) + 4 * (size_t)nnzb + 2 * 128 * (size_t)nnzb +
               8 * 4 * (size_t)nbr + 8 * (size_t)nnzb;           // rp ci H S diag(S) transpose map
    if (prec == MARNOLDI_MIXED) b += 2 * 128 * (size_t)nnzb;     // hi/lo FP32 copies of H and S
    return b + kScratchBytes;                                   // reduction scratch
}

size_t cells_bytes(int64_t nbr, const double *box)
{
    int64_t ncells = 1;
    for (int d = 0; d < 3; ++d) ncells *= (int64_t)std::max(1.0, std::min(256.0, std::floor(box[d] / 2.6)));
    return 24 * (size_t)nbr + 24 + 4 * (size_t)(ncells + 1) + 4 * (size_t)nbr;
}

// The solved columns [c0, c1) as a column state of their own (P stays shared:
// p_off holds absolute offsets).
ColumnState column_view(const ColumnState &st, int64_t c0, int64_t c1)
{
    ColumnState v = st;
    v.ncols = c1 - c0;
    v.cols = st.cols + c0;
    v.p_off = st.p_off + c0;
    v.nu_eff = st.nu_eff + c0;
    v.eig_status = st.eig_status + c0;
    v.eps = st.eps + c0 * st.nu;
    v.w = st.w + c0 * st.nu;
    v.t = st.t + c0 * st.nu;
    return v;
}

void free_state(marnoldi_ctx *c)
{
    if (c->state) dfree(c, c->state, c->state_bytes);
    c->state = nullptr;
    c->state_bytes = 0;
    c->solved = false;
}

}  // namespace

// ===================================================================== C ABI

extern "C" {

int marnoldi_set_allocator(marnoldi_alloc_fn alloc, marnoldi_free_fn free_fn, void *user)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return MARNOLDI_EINVAL;
    g_alloc = alloc;
    g_free = free_fn;
    g_user = user;
    return MARNOLDI_OK;
}

int marnoldi_kernel_kinds(void) { return KK_NKINDS; }

const char *marnoldi_last_error(const marnoldi_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_setup_err.c_str();
}

void marnoldi_destroy(marnoldi_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_state(c);
    if (c->ws) dfree(c, c->ws, c->ws_bytes);
    for (auto &p : c->owned) dfree(c, p.first, p.second);
    pinned_release(c->h_out);
    for (auto &p : c->pending) {
        c->events.push_back(p.second.first);
        c->events.push_back(p.second.second);
    }
    for (auto e : c->events) cudaEventDestroy(e);
    if (c->kexec) cudaGraphExecDestroy(c->kexec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    delete c;
}

int marnoldi_setup(marnoldi_ctx **out, int64_t n_block_rows, const int64_t *row_ptr,
                   const int32_t *col_idx, const double *H_vals, const double *S_vals,
                   const uint8_t *orbital_mask, const double *positions, const double *box,
                   int precision, void *cuda_stream)
{
    return setup_with_allocator(out, n_block_rows, row_ptr, col_idx, H_vals, S_vals, orbital_mask,
                                positions, box, precision, cuda_stream, g_alloc, g_free, g_user);
}

int marnoldi_device_bytes(const marnoldi_ctx *c, size_t *current, size_t *peak)
{
    if (!c) return MARNOLDI_EINVAL;
    if (current) *current = c->dev_bytes;
    if (peak) *peak = c->dev_peak;
    return MARNOLDI_OK;
}

int marnoldi_footprint(int64_t n_block_rows, const int64_t *row_ptr, const uint8_t *orbital_mask,
                       const double *box, int precision, int nu, int region_atoms,
                       int64_t batch_columns, size_t *bytes, int64_t *batch_used)
{
    g_setup_err.clear();
    if (!bytes) return fail(nullptr, MARNOLDI_EINVAL, "bytes is NULL");
    if (n_block_rows < 1 || n_block_rows > (int64_t)1 << 30 || !row_ptr)
        return fail(nullptr, MARNOLDI_EINVAL, "need n_block_rows >= 1 and row_ptr");
    PatternStats st;
    const int rc = pattern_stats(n_block_rows, row_ptr, orbital_mask, st);
    if (rc) return rc;
    return footprint_of(st, precision, nu, region_atoms, box, batch_columns, bytes, batch_used);
}

}  // extern "C"

int marnoldi::pattern_stats(int64_t n_block_rows, const int64_t *row_ptr, const uint8_t *orbital_mask,
                            PatternStats &st)
{
    st = PatternStats{};
    st.nbr = n_block_rows;
    st.nnzb = row_ptr[n_block_rows];
    st.m_vec = 4 * n_block_rows;
    for (int64_t I = 0; I < n_block_rows; ++I) {
        const int64_t len = row_ptr[I + 1] - row_ptr[I];
        if (len < 1) return fail(nullptr, MARNOLDI_EINVAL, "block row %lld is empty", (long long)I);
        st.maxrow = std::max<int>(st.maxrow, (int)len);
        for (int a = 0; a < 4; ++a)
            if (!orbital_mask || orbital_mask[4 * I + a]) {
                ++st.nc;
                st.prow += 4 * len;
            }
    }
    if (st.nc < 1) return fail(nullptr, MARNOLDI_EINVAL, "no real orbitals");
    return MARNOLDI_OK;
}

int marnoldi::footprint_of(const PatternStats &st, int precision, int nu, int region_atoms, const double *box,
                           int64_t batch_columns, size_t *bytes, int64_t *batch_used)
{
    if (precision != MARNOLDI_FP64 && precision != MARNOLDI_MIXED)
        return fail(nullptr, MARNOLDI_EINVAL, "unknown precision %d", precision);
    if (batch_columns < 1) return fail(nullptr, MARNOLDI_EINVAL, "batch_columns must be >= 1");
    const bool regional = region_atoms > 0;
    if (region_atoms < 0 || region_atoms > kMaxRegion || region_atoms > st.nbr || (regional && !box))
        return fail(nullptr, MARNOLDI_EINVAL, "region_atoms = %d invalid (regional mode needs box)", region_atoms);
    if (!regional && 4 * st.nbr > kMaxGlobalM)
        return fail(nullptr, MARNOLDI_EINVAL, "global mode supports M <= %lld", (long long)kMaxGlobalM);
    if (nu < 1 || nu > kMaxNu || (regional && nu > 4 * region_atoms))
        return fail(nullptr, MARNOLDI_EINVAL, "nu = %d out of range", nu);
    const int64_t B = clamp_batch(batch_columns, st.nc, regional);
    SolvePlan plan;
    if (!plan_solve(regional ? 4 * (int64_t)region_atoms : st.m_vec, precision, nu, region_atoms, st.maxrow,
                    st.nc, st.prow, B, regional ? 0 : (st.nbr + 7) / 8, plan))
        return fail(nullptr, MARNOLDI_EINVAL, "nu = %d exceeds the eigensolver's shared memory", nu);
    size_t total = setup_bytes(st.nbr, st.nnzb, precision) + plan.state_bytes + plan.ws_bytes +
                   (size_t)st.nnzb * 16 * sizeof(double) * 2;   // marnoldi_density's staging
    if (regional) total += cells_bytes(st.nbr, box);
    *bytes = total;
    if (batch_used) *batch_used = B;
    return MARNOLDI_OK;
}

int marnoldi::setup_with_allocator(marnoldi_ctx **out, int64_t n_block_rows, const int64_t *row_ptr,
                                   const int32_t *col_idx, const double *H_vals, const double *S_vals,
                                   const uint8_t *orbital_mask, const double *positions, const double *box,
                                   int precision, void *cuda_stream, marnoldi_alloc_fn alloc,
                                   marnoldi_free_fn free_fn, void *user)
{
    g_setup_err.clear();
    if (!out) return fail(nullptr, MARNOLDI_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_block_rows < 1) return fail(nullptr, MARNOLDI_EINVAL, "n_block_rows must be >= 1");
    if (!row_ptr || !col_idx || !H_vals || !S_vals) return fail(nullptr, MARNOLDI_EINVAL, "NULL matrix array");
    if (precision != MARNOLDI_FP64 && precision != MARNOLDI_MIXED)
        return fail(nullptr, MARNOLDI_EINVAL, "unknown precision %d", precision);
    if ((positions == nullptr) != (box == nullptr))
        return fail(nullptr, MARNOLDI_EINVAL, "positions and box must be given together");
    if (n_block_rows > (int64_t)1 << 30) return fail(nullptr, MARNOLDI_EINVAL, "too many block rows");
    const int64_t nnzb = row_ptr[n_block_rows];
    if (nnzb < n_block_rows || nnzb > ((int64_t)1 << 31) - 1)
        return fail(nullptr, MARNOLDI_EINVAL, "row_ptr[n_block_rows] = %lld is not a valid block count", (long long)nnzb);

    marnoldi_ctx *c = new marnoldi_ctx();
    {
        const char *g = getenv("MARNOLDI_KRYLOV_GRAPH");
        c->krylov_graph = g && g[0] == '1';
    }
    c->prec = precision;
    c->nbr = n_block_rows;
    c->nnzb = nnzb;
    c->m = 4 * n_block_rows;
    c->stream = (cudaStream_t)cuda_stream;
    c->alloc = alloc;
    c->free_fn = alloc ? free_fn : nullptr;
    c->user = user;
    c->rp.assign(row_ptr, row_ptr + n_block_rows + 1);
    c->ci.assign(col_idx, col_idx + nnzb);
    if (orbital_mask) {
        c->mask.assign(orbital_mask, orbital_mask + c->m);
        for (auto v : c->mask)
            if (v > 1) { delete c; return fail(nullptr, MARNOLDI_EINVAL, "orbital_mask values must be 0 or 1"); }
    }
    int rc = validate_structure(c, H_vals, S_vals);
    if (rc != MARNOLDI_OK) { delete c; return rc; }
    for (int64_t I = 0; I < n_block_rows; ++I)
        c->maxrow = std::max<int>(c->maxrow, (int)(c->rp[I + 1] - c->rp[I]));
    // transpose map: block (I, J) at k -> index of block (J, I)
    std::vector<int64_t> tmap(nnzb);
    for (int64_t I = 0; I < n_block_rows; ++I)
        for (int64_t k = c->rp[I]; k < c->rp[I + 1]; ++k) {
            const int64_t J = c->ci[k];
            const int32_t *b0 = c->ci.data() + c->rp[J], *b1 = c->ci.data() + c->rp[J + 1];
            tmap[k] = c->rp[J] + (std::lower_bound(b0, b1, (int32_t)I) - b0);
        }
    if (positions) {
        c->pos.assign(positions, positions + 3 * n_block_rows);
        c->box.assign(box, box + 3);
    }
    std::vector<double> sdiag(c->m, 1.0);
    for (int64_t I = 0; I < n_block_rows; ++I)
        for (int64_t k = c->rp[I]; k < c->rp[I + 1]; ++k)
            if (c->ci[k] == I)
                for (int a = 0; a < 4; ++a) sdiag[4 * I + a] = S_vals[16 * k + 5 * a];

    // ---- device upload
    int64_t *drp = nullptr, *dtm = nullptr;
    int32_t *dci = nullptr;
    double *dH = nullptr, *dS = nullptr, *dsd = nullptr;
    if ((rc = dupload(c, &drp, c->rp.data(), c->rp.size(), "row_ptr")) ||
        (rc = dupload(c, &dci, c->ci.data(), c->ci.size(), "col_idx")) ||
        (rc = dupload(c, &dH, H_vals, (size_t)16 * nnzb, "H")) ||
        (rc = dupload(c, &dS, S_vals, (size_t)16 * nnzb, "S")) ||
        (rc = dupload(c, &dsd, sdiag.data(), sdiag.size(), "diag S")) ||
        (rc = dupload(c, &dtm, tmap.data(), tmap.size(), "transpose map"))) {
        g_setup_err = c->err;
        marnoldi_destroy(c);
        return rc;
    }
    c->A.nbr = n_block_rows;
    c->A.nnzb = nnzb;
    c->A.rp = drp;
    c->A.ci = dci;
    c->A.Hd = dH;
    c->A.Sd = dS;
    c->A.sdiag = dsd;
    c->A.tmap = dtm;
    if (precision == MARNOLDI_MIXED) {
        // each block as 16 FP32 "hi" values then 16 "lo" values, hi + lo = the FP64 value
        std::vector<float> hf(32 * nnzb), sf(32 * nnzb);
        for (int64_t k = 0; k < nnzb; ++k)
            for (int q = 0; q < 16; ++q) {
                const double h = H_vals[16 * k + q], s = S_vals[16 * k + q];
                hf[32 * k + q] = (float)h;
                hf[32 * k + 16 + q] = (float)(h - (double)hf[32 * k + q]);
                sf[32 * k + q] = (float)s;
                sf[32 * k + 16 + q] = (float)(s - (double)sf[32 * k + q]);
            }
        float *dHf = nullptr, *dSf = nullptr;
        if ((rc = dupload(c, &dHf, hf.data(), hf.size(), "H fp32")) ||
            (rc = dupload(c, &dSf, sf.data(), sf.size(), "S fp32"))) {
            g_setup_err = c->err;
            marnoldi_destroy(c);
            return rc;
        }
        c->A.Hf = dHf;
        c->A.Sf = dSf;
    }
    // reduction scratch
    void *p = dalloc(c, kScratchBytes);
    if (!p) { g_setup_err = "device allocation failed"; marnoldi_destroy(c); return MARNOLDI_ENOMEM; }
    c->owned.push_back({p, kScratchBytes});
    c->d_partial = (double *)p;
    c->d_out = (double *)((char *)p + kOffOut);
    c->d_range = (double *)((char *)p + kOffRange);
    c->d_bisect = (BisectState *)((char *)p + kOffBisect);
    c->d_ticket = (unsigned *)((char *)p + kOffTicket);
    cudaError_t e = cudaMemsetAsync(p, 0, kScratchBytes, c->stream);
    if (e == cudaSuccess && !(c->h_out = pinned_slot())) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        fail_cuda(c, e, "setup");
        g_setup_err = c->err;
        marnoldi_destroy(c);
        return MARNOLDI_ECUDA;
    }
    *out = c;
    return MARNOLDI_OK;
}

extern "C" {

int marnoldi_set_batch(marnoldi_ctx *c, int64_t batch_columns)
{
    if (!c || batch_columns < 0) return MARNOLDI_EINVAL;
    c->batch_override = batch_columns;
    return MARNOLDI_OK;
}

int marnoldi_set_krylov_graph(marnoldi_ctx *c, int enable)
{
    if (!c || (enable != 0 && enable != 1)) return MARNOLDI_EINVAL;
    c->krylov_graph = enable == 1;
    return MARNOLDI_OK;
}

int marnoldi_krylov_graph_launches(const marnoldi_ctx *c, int64_t *graph_launches)
{
    if (!c || !graph_launches) return MARNOLDI_EINVAL;
    *graph_launches = c->graph_launches;
    return MARNOLDI_OK;
}

int marnoldi_set_profiling(marnoldi_ctx *c, int enable)
{
    if (!c) return MARNOLDI_EINVAL;
    c->profile = enable ? 1 : 0;
    return MARNOLDI_OK;
}

int marnoldi_kernel_stats(marnoldi_ctx *c, int kind, const char **name, int64_t *launches,
                          double *ms, int reset)
{
    if (!c || kind < 0 || kind >= KK_NKINDS) return MARNOLDI_EINVAL;
    if (name) *name = kernel_name(kind);
    if (launches) *launches = c->launches[kind];
    if (ms) *ms = c->ms[kind];
    if (reset) {
        c->launches[kind] = 0;
        c->ms[kind] = 0.0;
    }
    return MARNOLDI_OK;
}

int marnoldi_set_members(marnoldi_ctx *c, int n_members, const int64_t *atom_offsets,
                         const double *electron_counts)
{
    if (!c) return MARNOLDI_EINVAL;
    c->err.clear();
    c->solved = false;
    c->mem_atom.clear();
    c->mem_ne.clear();
    c->mem_kT.clear();
    c->mem_col.clear();
    if (n_members == 0) return MARNOLDI_OK;
    if (n_members < 0 || !atom_offsets || !electron_counts)
        return fail(c, MARNOLDI_EINVAL, "need n_members >= 0, atom_offsets and electron_counts");
    if (atom_offsets[0] != 0 || atom_offsets[n_members] != c->nbr)
        return fail(c, MARNOLDI_EINVAL, "atom_offsets must run from 0 to n_block_rows");
    for (int q = 0; q < n_members; ++q) {
        if (atom_offsets[q + 1] <= atom_offsets[q])
            return fail(c, MARNOLDI_EINVAL, "member %d is empty or the offsets descend", q);
        if (atom_offsets[q] % 8 != 0)
            return fail(c, MARNOLDI_EINVAL, "member %d starts at atom %lld, not a multiple of 8", q,
                        (long long)atom_offsets[q]);
        if (!(electron_counts[q] > 0.0) || !std::isfinite(electron_counts[q]))
            return fail(c, MARNOLDI_EINVAL, "member %d: electron count must be positive and finite", q);
        for (int64_t I = atom_offsets[q]; I < atom_offsets[q + 1]; ++I)
            for (int64_t k = c->rp[I]; k < c->rp[I + 1]; ++k)
                if (c->ci[k] < atom_offsets[q] || c->ci[k] >= atom_offsets[q + 1])
                    return fail(c, MARNOLDI_EINVAL, "block (%lld, %d) couples member %d to another member",
                                (long long)I, c->ci[k], q);
    }
    c->mem_atom.assign(atom_offsets, atom_offsets + n_members + 1);
    c->mem_ne.assign(electron_counts, electron_counts + n_members);
    return MARNOLDI_OK;
}

int marnoldi_set_member_temperatures(marnoldi_ctx *c, int n_members, const double *kT)
{
    if (!c) return MARNOLDI_EINVAL;
    c->err.clear();
    c->solved = false;
    if (c->mem_atom.empty() || n_members != (int)c->mem_atom.size() - 1 || !kT)
        return fail(c, MARNOLDI_EINVAL, "temperatures need the context's %d members",
                    c->mem_atom.empty() ? 0 : (int)c->mem_atom.size() - 1);
    for (int q = 0; q < n_members; ++q)
        if (!(kT[q] > 0.0) || !std::isfinite(kT[q]))
            return fail(c, MARNOLDI_EINVAL, "member %d: kT must be positive and finite", q);
    c->mem_kT.assign(kT, kT + n_members);
    return MARNOLDI_OK;
}

int marnoldi_member_energy(marnoldi_ctx *c, int member, double *band_energy, double *mu,
                           double *electron_count_out)
{
    if (!c) return MARNOLDI_EINVAL;
    if (!c->solved) return fail(c, MARNOLDI_ESTATE, "energy requested before a successful solve");
    if (c->mem_atom.empty() || member < 0 || member + 1 >= (int)c->mem_atom.size())
        return fail(c, MARNOLDI_EINVAL, "no member %d", member);
    if (band_energy) *band_energy = c->mem_E[member];
    if (mu) *mu = c->mem_mu[member];
    if (electron_count_out) *electron_count_out = c->mem_N[member];
    return MARNOLDI_OK;
}

int marnoldi_set_autotune(int mode)
{
    if (mode != 0 && mode != 1) return MARNOLDI_EINVAL;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_autotune = mode;
    return MARNOLDI_OK;
}

int marnoldi_check_status(int *compiled, int *site, int64_t *index)
{
    if (!compiled || !site || !index) return set_global_error(MARNOLDI_EINVAL, "check_status: NULL output");
    *compiled = kCheckBuild ? 1 : 0;
    *site = 0;
    *index = 0;
    cudaError_t (*take[])(unsigned long long *) = {check_take_krylov, check_take_region, check_take_outputs,
                                                   check_take_gs_stream};
    for (auto f : take) {
        unsigned long long w = 0;
        const cudaError_t e = f(&w);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_global_error(MARNOLDI_ECUDA, "check_status: reading the check words failed");
        }
        if (w && *site == 0) {
            *site = (int)((w >> 40) & 0x7fff);
            const unsigned long long lo = w & 0xffffffffffull;
            *index = (lo & (1ull << 39)) ? (int64_t)(lo | ~0xffffffffffull) : (int64_t)lo;
        }
    }
    return MARNOLDI_OK;
}

int marnoldi_gs_shape(const marnoldi_ctx *c, int *values_per_thread, int *threads)
{
    if (!c) return MARNOLDI_EINVAL;
    if (values_per_thread) *values_per_thread = c->gs_shape.vpt;
    if (threads) *threads = c->gs_shape.threads;
    return MARNOLDI_OK;
}

int marnoldi_solved_shape(marnoldi_ctx *c, int64_t *ncols, int *nu)
{
    if (!c) return MARNOLDI_EINVAL;
    if (!c->solved) return fail(c, MARNOLDI_ESTATE, "no solve yet");
    if (ncols) *ncols = c->ncols;
    if (nu) *nu = c->nu;
    return MARNOLDI_OK;
}

static int count_at(marnoldi_ctx *c, double mu, double kT, double *N, double *E)
{
    int rc = launch(c, KK_COUNT, [&] {
        return launch_count(c->st, mu, kT, c->d_partial, c->d_ticket, c->d_out, c->stream);
    });
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(c->h_out, c->d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e, "count read-back");
    if ((rc = sync(c, "count"))) return rc;
    *N = c->h_out[0];
    *E = c->h_out[1];
    return MARNOLDI_OK;
}

int marnoldi_solve(marnoldi_ctx *c, const int64_t *columns, int64_t ncols, int nu,
                   int region_atoms, double electron_count, double kT, const double *mu_fixed)
{
    if (!c) return MARNOLDI_EINVAL;
    const Phase phase("marnoldi_solve");
    c->err.clear();
    c->solved = false;   // a failed solve leaves no stale results
    const bool regional = region_atoms > 0;
    if (region_atoms < 0) return fail(c, MARNOLDI_EINVAL, "region_atoms must be >= 0");
    if (regional) {
        if (c->pos.empty())
            return fail(c, MARNOLDI_EINVAL, "regional mode needs positions and box at setup");
        if (region_atoms > c->nbr || region_atoms > kMaxRegion)
            return fail(c, MARNOLDI_EINVAL, "region_atoms = %d outside [1, min(n_block_rows, %d)]",
                        region_atoms, kMaxRegion);
    } else if (c->m > kMaxGlobalM) {
        return fail(c, MARNOLDI_EINVAL, "global mode supports M <= %lld (got %lld); use region_atoms > 0",
                    (long long)kMaxGlobalM, (long long)c->m);
    }
    if (!(kT > 0.0) || !std::isfinite(kT)) return fail(c, MARNOLDI_EINVAL, "kT must be positive and finite");
    if (mu_fixed && !std::isfinite(*mu_fixed)) return fail(c, MARNOLDI_EINVAL, "mu_fixed must be finite");
    const bool members = !c->mem_atom.empty();
    if (members) {
        // every member's own bisection, over its own columns, in global mode
        if (regional || columns || mu_fixed)
            return fail(c, MARNOLDI_EINVAL, "a solve of members takes every real orbital, global mode and "
                                            "a Fermi level by bisection");
        if (nu > 253)
            return fail(c, MARNOLDI_EINVAL, "a solve of members needs nu <= 253 (got %d)", nu);
    } else if (!mu_fixed && !(electron_count > 0.0 && std::isfinite(electron_count))) {
        return fail(c, MARNOLDI_EINVAL, "electron_count must be positive and finite");
    }
    // column list
    std::vector<int64_t> cols;
    if (!columns) {
        if (ncols >= 0) return fail(c, MARNOLDI_EINVAL, "columns is NULL but ncols >= 0");
        for (int64_t j = 0; j < c->m; ++j)
            if (c->mask.empty() || c->mask[j]) cols.push_back(j);
    } else {
        if (ncols < 1) return fail(c, MARNOLDI_EINVAL, "ncols must be >= 1");
        cols.assign(columns, columns + ncols);
        std::vector<int64_t> sorted = cols;
        std::sort(sorted.begin(), sorted.end());
        for (size_t q = 0; q < sorted.size(); ++q) {
            if (sorted[q] < 0 || sorted[q] >= c->m)
                return fail(c, MARNOLDI_EINVAL, "column %lld out of range", (long long)sorted[q]);
            if (q && sorted[q] == sorted[q - 1])
                return fail(c, MARNOLDI_EINVAL, "column %lld requested twice", (long long)sorted[q]);
            if (!c->mask.empty() && !c->mask[sorted[q]])
                return fail(c, MARNOLDI_EINVAL, "column %lld is a padding orbital", (long long)sorted[q]);
        }
    }
    if (cols.empty()) return fail(c, MARNOLDI_EINVAL, "no columns to solve");
    int64_t m_real = c->mask.empty() ? c->m : 0;
    if (!c->mask.empty())
        for (auto v : c->mask) m_real += v;
    if (nu < 1 || nu > kMaxNu || nu > m_real)
        return fail(c, MARNOLDI_EINVAL, "nu = %d outside [1, min(M_real = %lld, %d)]", nu, (long long)m_real, kMaxNu);
    if (regional && nu > 4 * region_atoms)
        return fail(c, MARNOLDI_EINVAL, "nu = %d exceeds the region's %d orbitals", nu, 4 * region_atoms);
    if (regional) {
        int rc0 = build_cells(c);
        if (rc0) return rc0;
        c->rm.n_reg = region_atoms;
    }

    free_state(c);
    const int64_t nc = (int64_t)cols.size();
    // per-column state: cols | p_off | nu_eff | eig_status | eps w t | P
    std::vector<int64_t> p_off(nc);
    int64_t prow = 0;
    for (int64_t q = 0; q < nc; ++q) {
        p_off[q] = prow * nu;
        const int64_t J = cols[q] >> 2;
        prow += 4 * (c->rp[J + 1] - c->rp[J]);
    }
    // vector length: the region, the largest member, or the structure
    int64_t m_vec = regional ? 4 * (int64_t)region_atoms : c->m;
    if (members) {
        m_vec = 0;
        for (size_t q = 0; q + 1 < c->mem_atom.size(); ++q)
            m_vec = std::max<int64_t>(m_vec, 4 * (c->mem_atom[q + 1] - c->mem_atom[q]));
    }
    const int64_t ntile_min = regional ? 0 : (c->nbr + 7) / 8;
    int64_t B = c->batch_override;
    if (B <= 0) {
        const ColumnShape shape = column_shape(m_vec, c->prec);
        const size_t per_col = per_column_bytes(shape, c->prec == 0 ? 8 : 4, nu, region_atoms, c->maxrow);
        size_t freeb = 0, totb = 0;
        if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess) { cudaGetLastError(); freeb = (size_t)8 << 30; }
        const size_t budget = std::min<size_t>(freeb / 2, (size_t)48 << 30);
        B = std::max<int64_t>(1, (int64_t)(budget / per_col));
    }
    B = clamp_batch(B, nc, regional);
    SolvePlan plan;
    if (!plan_solve(m_vec, c->prec, nu, region_atoms, c->maxrow, nc, prow, B, ntile_min, plan))
        return fail(c, MARNOLDI_EINVAL, "nu = %d with %d blocks per row exceeds the eigensolver's shared memory",
                    nu, c->maxrow);
    c->last_batch = B;
    c->state = dalloc(c, plan.state_bytes);
    if (!c->state)
        return fail(c, MARNOLDI_ENOMEM, "device allocation of %zu bytes for column state failed", plan.state_bytes);
    c->state_bytes = plan.state_bytes;
    char *sb = (char *)c->state;
    c->d_cols = (int64_t *)(sb + plan.o_cols);
    c->st.ncols = nc;
    c->st.nu = nu;
    c->st.cols = c->d_cols;
    c->st.p_off = (const int64_t *)(sb + plan.o_poff);
    c->st.nu_eff = (int *)(sb + plan.o_nue);
    c->st.eig_status = (int *)(sb + plan.o_est);
    c->st.eps = (double *)(sb + plan.o_eps);
    c->st.w = (double *)(sb + plan.o_w);
    c->st.t = (double *)(sb + plan.o_t);
    c->st.P = (double *)(sb + plan.o_P);
    cudaError_t e = cudaMemcpyAsync(c->d_cols, cols.data(), nc * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)c->st.p_off, p_off.data(), nc * 8, cudaMemcpyHostToDevice, c->stream);
    // regional product groups per batch: runs of one atom's columns, at most
    // regional_group() long, then the batch's column count as an end mark
    std::vector<int> grp;
    std::vector<int64_t> gofs;
    if (regional) {
        const int G = regional_group(c->prec);
        for (int64_t start = 0; start < nc; start += B) {
            const int64_t nbat = std::min<int64_t>(B, nc - start);
            gofs.push_back((int64_t)grp.size());
            for (int64_t q = 0; q < nbat;) {
                grp.push_back((int)q);
                const int64_t J = cols[start + q] >> 2;
                int64_t len = 1;
                while (q + len < nbat && len < G && (cols[start + q + len] >> 2) == J) ++len;
                q += len;
            }
            grp.push_back((int)nbat);
        }
        gofs.push_back((int64_t)grp.size());
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sb + plan.o_grp, grp.data(), grp.size() * 4, cudaMemcpyHostToDevice, c->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->st.eig_status, 0, nc * 4, c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e, "column state upload");

    // batch workspace
    const ColumnShape shape = plan.shape;
    const size_t vs = plan.vs;
    const size_t wtot = plan.ws_bytes;
    if (c->ws_bytes < wtot) {
        if (c->ws) dfree(c, c->ws, c->ws_bytes);
        c->ws = dalloc(c, wtot);
        c->ws_bytes = c->ws ? wtot : 0;
        if (!c->ws) return fail(c, MARNOLDI_ENOMEM, "device allocation of %zu bytes for the batch workspace failed", wtot);
    }
    // zero once: padding rows of the vectors must stay zero
    e = cudaMemsetAsync(c->ws, 0, wtot, c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e, "workspace clear");
    char *wb = (char *)c->ws;
    KrylovBatch kb{};
    kb.prec = c->prec;
    kb.nu = nu;
    kb.shape = shape;
    kb.K = wb + plan.oK;
    kb.SK = wb + plan.oSK;
    kb.U = wb + plan.oU;
    kb.Ulo = c->prec == 1 ? (void *)(wb + plan.oUl) : nullptr;
    kb.Hsub = (double *)(wb + plan.oH);
    kb.Lsub = (double *)(wb + plan.oL);
    kb.scale = (double *)(wb + plan.oSc);
    kb.cn2 = (double *)(wb + plan.oC);
    kb.status = (int *)(wb + plan.oS);
    kb.nu_eff = (int *)(wb + plan.oN);
    kb.m = m_vec;
    kb.ntile = (int)plan.ntile;
    kb.thop = (uint8_t *)(wb + plan.oTh);
    kb.tinv = (uint16_t *)(wb + plan.oTo);
    kb.tcnt = (int *)(wb + plan.oTc);
    EigScratch es = plan.es;
    es.D = (double *)(wb + plan.oED);
    es.E = (double *)(wb + plan.oEE);
    es.RQ = (double *)(wb + plan.oERQ);
    es.rot = (double2 *)(wb + plan.oERot);
    es.sweep = (int2 *)(wb + plan.oESw);
    es.nsweep = (int *)(wb + plan.oENs);
    es.Ag = plan.a_global ? (double *)(wb + plan.oEA) : nullptr;
    RegionMaps *rmp = nullptr;
    if (regional) {
        c->rm.reg = (int *)(wb + plan.oRg);
        c->rm.lcnt = (int *)(wb + plan.oRc);
        c->rm.lci = (int *)(wb + plan.oRi);
        c->rm.lgk = (int *)(wb + plan.oRk);
        c->rm.rstat = (int *)(wb + plan.oRs);
        rmp = &c->rm;
    }
    const double tau = c->prec == 0 ? kTauFp64 : kTauMixed;
    const int64_t mp = shape.m_pad;
    int rc = MARNOLDI_OK;
    // the Krylov build of one batch (the vectors are stored in the tile order
    // that the support search sets); slot n holds w_n (unnormalised); H w_n
    // goes to U and, for n >= 1, S w_n to its slot (S w_0 comes from the
    // initialisation); the Gram-Schmidt of step n scales them and writes w_{n+1}
    auto build = [&](const KrylovBatch &k) -> int {
        int r;
        if ((r = launch(c, KK_SUPPORT, [&] { return launch_support(c->A, rmp, k, c->stream); })))
            return r;
        const int rows = regional ? region_atoms : (int)c->nbr;
        if ((rows & 7) && (r = launch(c, KK_INIT, [&] { return launch_zero_partial_tile(k, rows, c->stream); })))
            return r;
        if ((r = launch(c, KK_INIT, [&] {
                 return regional ? launch_init_regional(c->A, c->rm, k, c->stream) : launch_init(c->A, k, c->stream);
             })))
            return r;
        for (int n = 0; n < nu; ++n) {
            const char *Kn = (const char *)k.K + (size_t)n * mp * vs;
            char *SKn = n > 0 ? (char *)k.SK + (size_t)n * mp * vs : nullptr;
            if (regional) {
                if ((r = launch(c, KK_SPMM_HS, [&] {
                         return launch_spmm_regional_hs(c->A, c->rm, k, Kn, (int64_t)nu * mp, SKn,
                                                        (int64_t)nu * mp, n + 1, c->stream);
                     })))
                    return r;
            } else if ((r = launch(c, KK_SPMM_HS, [&] {
                            return launch_spmm_hs(c->A, k, Kn, (int64_t)nu * mp, SKn, (int64_t)nu * mp, n + 1,
                                                  c->stream);
                        }))) {
                return r;
            }
            if ((r = launch(c, KK_GS, [&] { return launch_gs(k, n, n + 1 < nu, tau, c->stream); })))
                return r;
        }
        return MARNOLDI_OK;
    };
    // projection scratch (batch columns x nu) while proj_vec is set
    DeviceBuffer proj_buf(c, c->proj_vec ? (size_t)B * nu * sizeof(double) : 0);
    if (c->proj_vec && !proj_buf.get()) return fail(c, MARNOLDI_ENOMEM, "device allocation for the projection failed");
    const TuneKey key{c->prec, nu, regional ? 1 : 0, mp};
    bool tune = false;
    if (autotune_mode()) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        load_tune_cache_locked();
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) kb.shape = it->second;
        else tune = true;
    }
    for (int64_t start = 0; start < nc; start += B) {
        kb.nb = (int)std::min<int64_t>(B, nc - start);
        kb.cols = c->d_cols + start;
        if (regional) {
            const int64_t bi = start / B;
            c->rm.gstart = (const int *)(sb + plan.o_grp) + gofs[bi];
            c->rm.ngroups = (int)(gofs[bi + 1] - gofs[bi] - 1);
            const Phase ph("region");
            if ((rc = find_regions(c, kb))) return rc;
            if ((rc = launch(c, KK_REGION, [&] { return launch_local_bsr(c->A, c->rm, kb, c->stream); })))
                return rc;
        }
        if (tune) {
            // time every shape on the batch's first columns (one run to warm
            // up, one timed) and keep the fastest for this key from now on;
            // the lock makes concurrent solves of the same key agree
            std::lock_guard<std::mutex> lock(g_tune_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                kb.shape = it->second;
            } else {
                ColumnShape cand[kMaxShapes];
                const int ncand = column_shape_candidates(mp, c->prec, cand);
                KrylovBatch ks = kb;
                ks.nb = (int)std::min<int64_t>(kb.nb, kTuneColumns);
                float best = 0.f;
                ColumnShape pick = kb.shape;
                cudaEvent_t e0 = get_event(c), e1 = get_event(c);
                for (int q = 0; q < ncand && ncand > 1; ++q) {
                    ks.shape = cand[q];
                    float ms = 0.f;
                    for (int rep = 0; rep < 2; ++rep) {
                        if (rep == 1) cudaEventRecord(e0, c->stream);
                        if ((rc = build(ks))) break;
                        if (rep == 1) cudaEventRecord(e1, c->stream);
                    }
                    if (rc || (rc = sync(c, "autotune"))) break;
                    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        cudaGetLastError();
                        continue;
                    }
                    if (q == 0 || ms < best) {
                        best = ms;
                        pick = cand[q];
                    }
                }
                c->events.push_back(e0);
                c->events.push_back(e1);
                if (rc) return rc;
                g_tuned[key] = pick;
                save_tune_entry_locked(key, pick);
                kb.shape = pick;
            }
            tune = false;
        }
        {
            const Phase ph("krylov");   // support search, initial vectors, nu steps of SpMM + Gram-Schmidt
            // as one graph when asked for (not while kernels are timed one by one)
            if ((rc = c->krylov_graph && !c->profile ? run_as_graph(c, [&] { return build(kb); }) : build(kb)))
                return rc;
        }
        if (c->proj_vec) {
            if ((rc = launch(c, KK_EIGSTATE, [&] {
                     return launch_project(kb, c->proj_vec, c->m, proj_buf.get(), c->stream);
                 })))
                return rc;
            es.proj = proj_buf.get();
            es.proj_out = c->proj_out;
        }
        const Phase ph("eigensolve");
        if ((rc = launch(c, KK_EIG, [&] { return launch_eig(c->A, kb, c->st, start, rmp, es, c->stream); })))
            return rc;
    }
    c->gs_shape = kb.shape;
    c->last_kb = kb;
    c->last_regional = regional;
    c->last_all_real = columns == nullptr;
    // ---- Fermi level
    const Phase ph_fermi("fermi");
    double mu = 0.0, N = 0.0, E = 0.0;
    if (mu_fixed) {
        mu = *mu_fixed;
        if ((rc = count_at(c, mu, kT, &N, &E))) return rc;
    } else {
        // level range and the whole bisection on the device, one read-back;
        // members: one bisection over each member's columns
        const size_t nmem = members ? c->mem_atom.size() - 1 : 1;
        std::vector<int64_t> col0(nmem + 1, 0);
        if (members) {
            size_t q = 0;
            for (size_t m = 0; m < nmem; ++m) {
                col0[m] = (int64_t)q;
                while (q < cols.size() && (cols[q] >> 2) < c->mem_atom[m + 1]) ++q;
            }
        }
        col0[nmem] = nc;
        std::vector<double> mmu(nmem), mN(nmem), mE(nmem);
        for (size_t m = 0; m < nmem; ++m) {
            const double ne = members ? c->mem_ne[m] : electron_count;
            const double mkT = members && !c->mem_kT.empty() ? c->mem_kT[m] : kT;
            const ColumnState sub = column_view(c->st, col0[m], col0[m + 1]);
            if (sub.ncols == 0)
                return fail(c, MARNOLDI_EINVAL, "member %zu has no real orbitals", m);
            if ((rc = launch(c, KK_COUNT, [&] {
                     return launch_bisection(sub, mkT, ne, c->d_partial, c->d_ticket, c->d_range, c->d_out,
                                             c->d_bisect, c->stream);
                 })))
                return rc;
            e = cudaMemcpyAsync(c->h_out, c->d_bisect, sizeof(BisectState), cudaMemcpyDeviceToHost, c->stream);
            if (e != cudaSuccess) return fail_cuda(c, e, "bisection read-back");
            if ((rc = sync(c, "bisection"))) return rc;
            BisectState bs;
            memcpy(&bs, c->h_out, sizeof bs);
            // one launch each of the range and of the graph was counted; add the
            // loop's kernels (a step and a count per iteration)
            c->launches[KK_MINMAX] += 1;
            c->launches[KK_COUNT] += bs.steps - 1;
            c->launches[KK_BISECT] += bs.steps;
            if (bs.status == 1)
                return fail(c, MARNOLDI_ENOCONV, "electron count %.6g outside [N(lo) = %.6g, N(hi) = %.6g]%s",
                            ne, bs.Nlo, bs.Nhi, members ? " for a member" : "");
            mmu[m] = bs.mu;
            mN[m] = bs.N;
            mE[m] = bs.E;
            N += bs.N;
            E += bs.E;
        }
        mu = mmu[0];
        if (members) {
            c->mem_col = col0;
            c->mem_mu = mmu;
            c->mem_N = mN;
            c->mem_E = mE;
        }
    }
    if ((rc = sync(c, "solve"))) return rc;
    std::vector<int> est(nc);
    e = cudaMemcpyAsync(est.data(), c->st.eig_status, nc * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e, "status read-back");
    if ((rc = sync(c, "status read-back"))) return rc;
    c->ncols = nc;
    c->nu = nu;
    c->cols = std::move(cols);
    c->mu = mu;
    c->N = N;
    c->E = E;
    c->kT = kT;
    c->solved = true;
    for (int64_t q = 0; q < nc; ++q) {
        if (est[q] & 4)
            return fail(c, MARNOLDI_ETIMEOUT, "column %lld: a bounded wait of the Gram-Schmidt kernel gave up",
                        (long long)c->cols[q]);
        if (est[q] & 2)
            return fail(c, MARNOLDI_ENOTSPD, "column %lld: a Krylov vector has non-positive S norm", (long long)c->cols[q]);
        if (est[q] & 1)
            return fail(c, MARNOLDI_ENOCONV, "column %lld: QL iteration did not converge", (long long)c->cols[q]);
    }
    return MARNOLDI_OK;
}

int marnoldi_density_device(marnoldi_ctx *c, double *rho, double *rhoE)
{
    const Phase phase("density");
    if (!c || !rho || !rhoE) return MARNOLDI_EINVAL;
    if (!c->solved) return fail(c, MARNOLDI_ESTATE, "density requested before a successful solve");
    const size_t bytes = (size_t)c->nnzb * 16 * sizeof(double);
    cudaError_t e = cudaMemsetAsync(rho, 0, bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(rhoE, 0, bytes, c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e, "density clear");
    if (c->mem_atom.empty())
        return launch(c, KK_DENSITY, [&] {
            return launch_density(c->A, c->st, c->mu, c->kT, rho, rhoE, c->stream);
        });
    for (size_t m = 0; m + 1 < c->mem_col.size(); ++m) {   // each member at its own Fermi level
        const ColumnState sub = column_view(c->st, c->mem_col[m], c->mem_col[m + 1]);
        const int rc = launch(c, KK_DENSITY, [&] {
            return launch_density(c->A, sub, c->mem_mu[m], c->mem_kT.empty() ? c->kT : c->mem_kT[m], rho, rhoE,
                                  c->stream);
        });
        if (rc) return rc;
    }
    return MARNOLDI_OK;
}

int marnoldi_density(marnoldi_ctx *c, double *rho, double *rhoE)
{
    if (!c || !rho || !rhoE) return MARNOLDI_EINVAL;
    if (!c->solved) return fail(c, MARNOLDI_ESTATE, "density requested before a successful solve");
    const size_t bytes = (size_t)c->nnzb * 16 * sizeof(double);
    double *d = (double *)dalloc(c, 2 * bytes);
    if (!d) return fail(c, MARNOLDI_ENOMEM, "device allocation for density output failed");
    int rc = marnoldi_density_device(c, d, d + c->nnzb * 16);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = cudaMemcpyAsync(rho, d, bytes, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(rhoE, d + c->nnzb * 16, bytes, cudaMemcpyDeviceToHost, c->stream);
    }
    dfree(c, d, 2 * bytes);
    if (!rc && e != cudaSuccess) rc = fail_cuda(c, e, "density read-back");
    int rs = sync(c, "density");
    return rc ? rc : rs;
}

int marnoldi_energy(marnoldi_ctx *c, double *band_energy, double *mu, double *electron_count_out)
{
    if (!c) return MARNOLDI_EINVAL;
    if (!c->solved) return fail(c, MARNOLDI_ESTATE, "energy requested before a successful solve");
    if (band_energy) *band_energy = c->E;
    if (mu) *mu = c->mu;
    if (electron_count_out) *electron_count_out = c->N;
    return MARNOLDI_OK;
}

int marnoldi_level_range(marnoldi_ctx *c, double *eps_min, double *eps_max)
{
    if (!c || !eps_min || !eps_max) return MARNOLDI_EINVAL;
    if (!c->solved) return fail(c, MARNOLDI_ESTATE, "level range requested before a successful solve");
    if (!c->mem_atom.empty()) return fail(c, MARNOLDI_EINVAL, "level range of a context with members");
    int rc = launch(c, KK_MINMAX, [&] {
        return launch_minmax(c->st, c->d_partial, c->d_ticket, c->d_out, c->stream);
    });
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(c->h_out, c->d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e, "minmax read-back");
    if ((rc = sync(c, "minmax"))) return rc;
    *eps_min = c->h_out[0];
    *eps_max = c->h_out[1];
    return MARNOLDI_OK;
}

int marnoldi_fermi_at(marnoldi_ctx *c, double mu, double kT, double *N, double *E)
{
    if (!c || !(kT > 0.0) || !std::isfinite(mu) || !std::isfinite(kT)) return MARNOLDI_EINVAL;
    if (!c->solved) return fail(c, MARNOLDI_ESTATE, "Fermi level set before a successful solve");
    if (!c->mem_atom.empty()) return fail(c, MARNOLDI_EINVAL, "one Fermi level for a context with members");
    double n = 0.0, en = 0.0;
    const int rc = count_at(c, mu, kT, &n, &en);
    if (rc) return rc;
    c->mu = mu;
    c->kT = kT;
    c->N = n;
    c->E = en;
    if (N) *N = n;
    if (E) *E = en;
    return MARNOLDI_OK;
}

int marnoldi_green(marnoldi_ctx *c, const double *z, int nz, double *G)
{
    const Phase phase("green");
    if (!c || (nz > 0 && (!z || !G)) || nz < 0) return MARNOLDI_EINVAL;
    if (!c->solved) return fail(c, MARNOLDI_ESTATE, "green requested before a successful solve");
    const size_t per = (size_t)c->nnzb * 16 * 2;
    double *d = (double *)dalloc(c, per * sizeof(double));
    if (!d) return fail(c, MARNOLDI_ENOMEM, "device allocation for green output failed");
    int rc = MARNOLDI_OK;
    for (int q = 0; q < nz && !rc; ++q) {
        if (!std::isfinite(z[2 * q]) || !std::isfinite(z[2 * q + 1]) || z[2 * q + 1] == 0.0) {
            rc = fail(c, MARNOLDI_EINVAL, "shift %d must be finite with a nonzero imaginary part", q);
            break;
        }
        cudaError_t e = cudaMemsetAsync(d, 0, per * sizeof(double), c->stream);
        if (e != cudaSuccess) { rc = fail_cuda(c, e, "green clear"); break; }
        rc = launch(c, KK_GREEN, [&] {
            return launch_green(c->A, c->st, z[2 * q], z[2 * q + 1], d, c->stream);
        });
        if (rc) break;
        e = cudaMemcpyAsync(G + q * per, d, per * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) rc = fail_cuda(c, e, "green read-back");
    }
    dfree(c, d, per * sizeof(double));
    int rs = sync(c, "green");
    return rc ? rc : rs;
}

int marnoldi_forces(marnoldi_ctx *c, const double *dH, const double *dS, double *F)
{
    const Phase phase("forces");
    if (!c || !dH || !dS || !F) return MARNOLDI_EINVAL;
    if (!c->solved) return fail(c, MARNOLDI_ESTATE, "forces requested before a successful solve");
    const size_t vals = (size_t)c->nnzb * 16, bytes = (size_t)(2 + 6) * vals * sizeof(double) +
                                                      (size_t)c->nbr * 3 * sizeof(double);
    double *d = (double *)dalloc(c, bytes);
    if (!d) return fail(c, MARNOLDI_ENOMEM, "device allocation of %zu bytes for forces failed", bytes);
    double *rho = d, *rhoE = d + vals, *dHd = d + 2 * vals, *dSd = d + 5 * vals, *Fd = d + 8 * vals;
    int rc = marnoldi_density_device(c, rho, rhoE);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = cudaMemcpyAsync(dHd, dH, 3 * vals * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dSd, dS, 3 * vals * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) rc = fail_cuda(c, e, "force inputs upload");
    }
    if (!rc)
        rc = launch(c, KK_FORCE, [&] { return launch_forces(c->A, rho, rhoE, dHd, dSd, Fd, c->stream); });
    if (!rc) {
        e = cudaMemcpyAsync(F, Fd, (size_t)c->nbr * 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) rc = fail_cuda(c, e, "force read-back");
    }
    const int rs = sync(c, "forces");
    dfree(c, d, bytes);
    return rc ? rc : rs;
}

int marnoldi_eigenstate(marnoldi_ctx *c, int64_t k, double sigma, double *eps_k, double *phi,
                        double *eta_bounds)
{
    if (!c || !eps_k || !phi) return MARNOLDI_EINVAL;
    const Phase phase("eigenstate");
    if (!c->solved) return fail(c, MARNOLDI_ESTATE, "eigenstate requested before a successful solve");
    if (!c->mem_atom.empty() || c->last_regional || !c->last_all_real)
        return fail(c, MARNOLDI_EINVAL, "the eigenstate needs a global-mode solve of every real orbital "
                                        "of one structure");
    if (c->nu > eigvec_max_nu())
        return fail(c, MARNOLDI_EINVAL, "the eigenstate supports nu <= %d (got %d)", eigvec_max_nu(), c->nu);
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(c, MARNOLDI_EINVAL, "sigma must be positive and finite");
    const int64_t m_real = c->ncols;
    if (k < 1 || k > m_real)
        return fail(c, MARNOLDI_EINVAL, "k = %lld outside [1, %lld]", (long long)k, (long long)m_real);
    // eta(n): the inverse integrated density of states, by the bisection on
    // the level count (which carries the spin factor 2, so N = 2 n)
    auto eta = [&](double n, double *out) -> int {
        if (n <= 0.0) { *out = -INFINITY; return MARNOLDI_OK; }
        if (n >= (double)m_real) { *out = INFINITY; return MARNOLDI_OK; }
        int rc = launch(c, KK_COUNT, [&] {
            return launch_bisection(c->st, sigma, 2.0 * n, c->d_partial, c->d_ticket, c->d_range, c->d_out,
                                    c->d_bisect, c->stream);
        });
        if (rc) return rc;
        cudaError_t e = cudaMemcpyAsync(c->h_out, c->d_bisect, sizeof(BisectState), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return fail_cuda(c, e, "bisection read-back");
        if ((rc = sync(c, "eigenstate bisection"))) return rc;
        BisectState bs;
        memcpy(&bs, c->h_out, sizeof bs);
        c->launches[KK_MINMAX] += 1;
        c->launches[KK_COUNT] += bs.steps - 1;
        c->launches[KK_BISECT] += bs.steps;
        if (bs.status == 1) return fail(c, MARNOLDI_ENOCONV, "n = %.6g outside the bracket of the levels", n);
        *out = bs.mu;
        return MARNOLDI_OK;
    };
    double lo, ek, hi;
    int rc;
    if ((rc = eta((double)k - 1.0, &lo)) || (rc = eta((double)k - 0.5, &ek)) || (rc = eta((double)k, &hi))) return rc;
    const int64_t nc = c->ncols, M = c->m;
    const int nu = c->nu;
    // the weights of the window and the reference (column, level)
    DeviceBuffer wbuf(c, (size_t)nc * (sizeof(double) + sizeof(int)) + 16);
    if (!wbuf.get()) return fail(c, MARNOLDI_ENOMEM, "device allocation for the eigenstate failed");
    double *colmax = wbuf.get();
    int *colarg = (int *)(colmax + nc);
    int64_t *argmax = (int64_t *)(((uintptr_t)(colarg + nc) + 7) & ~(uintptr_t)7);
    if ((rc = launch(c, KK_EIGSTATE, [&] {
             return launch_window(c->st, lo, hi, sigma, colmax, colarg, argmax, c->stream);
         })))
        return rc;
    std::vector<double> hmax(nc);
    std::vector<int> harg(nc);
    int64_t cstar = -1;
    cudaError_t e = cudaMemcpyAsync(hmax.data(), colmax, nc * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(harg.data(), colarg, nc * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cstar, argmax, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e, "eigenstate weights read-back");
    if ((rc = sync(c, "eigenstate weights"))) return rc;
    *eps_k = ek;
    if (eta_bounds) {
        eta_bounds[0] = lo;
        eta_bounds[1] = hi;
    }
    memset(phi, 0, (size_t)M * sizeof(double));
    if (cstar < 0 || !(hmax[cstar] > 0.0)) return MARNOLDI_OK;   // no weight in the window
    // columns whose contributions matter, in solved order
    std::vector<int64_t> sel;
    for (int64_t q = 0; q < nc; ++q)
        if (hmax[q] > 0.0 && hmax[q] >= 1e-12 * hmax[cstar]) sel.push_back(c->cols[q]);
    // a view of the structure with its own state and workspace: first the
    // reference column alone (its vector K v_a, from its batch's workspace),
    // then the selected columns with the projection on that vector
    marnoldi_ctx *v = new marnoldi_ctx();
    v->stream = c->stream;
    v->prec = c->prec;
    v->nbr = c->nbr;
    v->nnzb = c->nnzb;
    v->m = c->m;
    v->maxrow = c->maxrow;
    v->rp = c->rp;
    v->ci = c->ci;
    v->mask = c->mask;
    v->alloc = c->alloc;
    v->free_fn = c->free_fn;
    v->user = c->user;
    v->A = c->A;
    v->shares_structure = true;
    v->batch_override = c->batch_override;
    auto done = [&](int code) {
        for (int q = 0; q < KK_NKINDS; ++q) {
            c->launches[q] += v->launches[q];
            c->ms[q] += v->ms[q];
        }
        if (code && c->err.empty()) c->err = v->err;
        marnoldi_destroy(v);
        return code;
    };
    {
        void *p = dalloc(v, kScratchBytes);
        if (!p) return done(fail(c, MARNOLDI_ENOMEM, "device allocation for the eigenstate failed"));
        v->owned.push_back({p, kScratchBytes});
        v->d_partial = (double *)p;
        v->d_out = (double *)((char *)p + kOffOut);
        v->d_range = (double *)((char *)p + kOffRange);
        v->d_bisect = (BisectState *)((char *)p + kOffBisect);
        v->d_ticket = (unsigned *)((char *)p + kOffTicket);
        e = cudaMemsetAsync(p, 0, kScratchBytes, v->stream);
        if (e != cudaSuccess) return done(fail_cuda(c, e, "eigenstate scratch"));
        if (!(v->h_out = pinned_slot())) return done(fail(c, MARNOLDI_ENOMEM, "pinned read-back slot"));
    }
    const double zero = 0.0;
    const int64_t jref = c->cols[cstar];
    if ((rc = marnoldi_solve(v, &jref, 1, nu, 0, 0.0, sigma, &zero))) return done(rc);
    double eref = 0.0;
    e = cudaMemcpyAsync(&eref, v->st.eps + harg[cstar], sizeof(double), cudaMemcpyDeviceToHost, v->stream);
    if (e != cudaSuccess) return done(fail_cuda(c, e, "reference level read-back"));
    if ((rc = sync(v, "reference level"))) return done(rc);
    // buffers owned by the view, released with it
    auto vbuf = [&](size_t bytes) -> double * {
        void *q = dalloc(v, bytes);
        if (q) v->owned.push_back({q, bytes});
        return (double *)q;
    };
    double *vref = vbuf((size_t)M * sizeof(double));
    const size_t agb = eigvec_scratch_bytes(nu);
    double *ag = agb ? vbuf(agb) : nullptr;
    if (agb && !ag) return done(fail(c, MARNOLDI_ENOMEM, "eigenstate buffers"));
    double *proj = vbuf(sel.size() * (size_t)nu * sizeof(double));
    double *phid = vbuf((size_t)M * sizeof(double));
    if (!vref || !proj || !phid) return done(fail(c, MARNOLDI_ENOMEM, "eigenstate buffers"));
    e = cudaMemsetAsync(vref, 0, (size_t)M * sizeof(double), v->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(phid, 0, (size_t)M * sizeof(double), v->stream);
    if (e != cudaSuccess) return done(fail_cuda(c, e, "eigenstate buffers"));
    if ((rc = launch(v, KK_EIGSTATE, [&] { return launch_eigvec(v->last_kb, 0, eref, M, vref, ag, v->stream); })))
        return done(rc);
    v->proj_vec = vref;
    v->proj_out = proj;
    rc = marnoldi_solve(v, sel.data(), (int64_t)sel.size(), nu, 0, 0.0, sigma, &zero);
    v->proj_vec = nullptr;
    v->proj_out = nullptr;
    if (rc) return done(rc);
    if ((rc = launch(v, KK_EIGSTATE, [&] {
             return launch_combine(v->st, proj, lo, hi, sigma, phid, v->stream);
         })))
        return done(rc);
    e = cudaMemcpyAsync(phi, phid, (size_t)M * sizeof(double), cudaMemcpyDeviceToHost, v->stream);
    if (e != cudaSuccess) return done(fail_cuda(c, e, "eigenvector read-back"));
    rc = sync(v, "eigenvector");
    return done(rc);
}

int marnoldi_column_stats(marnoldi_ctx *c, int32_t *nu_eff, double *eps, double *w)
{
    if (!c) return MARNOLDI_EINVAL;
    if (!c->solved) return fail(c, MARNOLDI_ESTATE, "column stats requested before a successful solve");
    int rc = sync(c, "column stats");
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    const size_t n = (size_t)c->ncols * c->nu;
    if (nu_eff) e = cudaMemcpyAsync(nu_eff, c->st.nu_eff, c->ncols * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && eps) e = cudaMemcpyAsync(eps, c->st.eps, n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && w) e = cudaMemcpyAsync(w, c->st.w, n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return fail_cuda(c, e, "column stats read-back");
    return sync(c, "column stats read-back");
}

}  // extern "C"
