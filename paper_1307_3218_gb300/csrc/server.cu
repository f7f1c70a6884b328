// Request server over libmarnoldi: structures of different sizes and subspace
// dimensions arrive at any time and run concurrently on one GPU.
//
// Every request is a whole multiple Arnoldi calculation (arXiv:1307.3218,
// Section 2): setup of its (H, S), the Krylov subspaces of all real orbitals,
// their eigensolves, the Fermi level by bisection, and the density and
// energy-density matrices.  Worker threads each own a non-blocking CUDA stream
// and take requests from one FIFO queue; the kernels of requests that run at
// the same time share the GPU (a small structure fills a few SMs, so its
// launches overlap with those of a large one).  A request is admitted when its
// device-memory footprint (marnoldi_footprint: structure, column state, batch
// workspace and density staging) fits under the server's budget beside the
// requests already running; its batch size is chosen so that the footprint
// stays within budget / workers when possible.  All device memory comes from
// one memory pool of the server that keeps freed memory mapped, so requests
// reuse it without new mappings; a request's H, S and Krylov state stay
// resident from its setup to its last read-back.
//
// Continuous batching: when a worker starts a request, queued requests of the
// same precision, nu and kT whose Krylov vectors have the same padded length
// join it as members of one block-diagonal union (marnoldi_set_members), so
// that one launch per step covers all their columns, as long as the union's
// footprint fits.
//
// Results do not depend on the mix: a request's kernels see only its own
// data, its batch size changes which columns share a launch but not any
// column's arithmetic, its reductions run in a fixed order, and as a member of
// a union it keeps its own tile order, launch shape and Fermi level.
#include "marnoldi.h"
#include "internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

thread_local std::string t_server_err;

// Requests of one precision and nu whose Krylov vectors have the same padded
// length run as members of one context (a block-diagonal union, one launch
// per step for all of them) when they wait in the queue together: at most
// kDefaultGroup members and 4,096 atoms (the global-mode limit) per union.
constexpr int kDefaultGroup = 16;
constexpr int64_t kGroupAtoms = 4096;

int server_fail(int code, const char *msg)
{
    t_server_err = msg;
    return code;
}

struct Request {
    int64_t id = 0;
    // inputs (caller-owned until the request has been waited for)
    int64_t nbr = 0;
    const int64_t *rp = nullptr;
    const int32_t *ci = nullptr;
    const double *H = nullptr, *S = nullptr;
    const uint8_t *mask = nullptr;
    const double *pos = nullptr, *box = nullptr;
    int prec = 0, nu = 0, region_atoms = 0;
    double electron_count = 0.0, kT = 0.0;
    double *rho = nullptr, *rhoE = nullptr;
    int64_t batch = 0;
    size_t bytes = 0;
    marnoldi::PatternStats stats;   // of the block pattern, for footprints of groups
    int64_t m_pad = 0;              // padded vector length alone
    // results
    bool done = false;
    int status = MARNOLDI_OK;
    std::string msg;
    double E = 0.0, mu = 0.0, N = 0.0;
    double t_submit = 0.0, t_start = 0.0, t_end = 0.0;
};

}  // namespace

struct marnoldi_server {
    std::mutex mu;
    std::condition_variable cv_admit, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
    size_t budget = 0, in_use = 0, peak = 0;
    int workers = 0, running = 0, peak_running = 0;
    int max_group = kDefaultGroup;
    int64_t next_id = 1, completed = 0, groups = 0, largest_group = 1;
    bool stopping = false;
    int device = 0;
    cudaMemPool_t pool = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<std::thread> threads;
    std::chrono::steady_clock::time_point t0;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void *pool_alloc(size_t bytes, void *stream, void *user)
{
    auto *srv = (marnoldi_server *)user;
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, srv->pool, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pool_free(void *p, size_t, void *stream, void *)
{
    cudaFreeAsync(p, (cudaStream_t)stream);
}

// Footprint and batch of a pattern: the caller's batch, else the largest whose
// footprint stays within `share` (at least one column).
int choose_batch(const marnoldi::PatternStats &st, int prec, int nu, int region_atoms, const double *box,
                 int64_t batch_columns, size_t share, size_t *bytes, int64_t *used)
{
    using marnoldi::footprint_of;
    if (batch_columns > 0) return footprint_of(st, prec, nu, region_atoms, box, batch_columns, bytes, used);
    int rc = footprint_of(st, prec, nu, region_atoms, box, (int64_t)1 << 40, bytes, used);
    if (rc || *bytes <= share) return rc;
    int64_t lo = 1, hi = *used;   // footprints grow with the batch
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        size_t b = 0;
        if ((rc = footprint_of(st, prec, nu, region_atoms, box, mid, &b, nullptr))) return rc;
        if (b <= share) lo = mid; else hi = mid - 1;
    }
    return footprint_of(st, prec, nu, region_atoms, box, lo, bytes, used);
}

// Atoms of a member in a union: its own, rounded up to 8 unless it is last.
int64_t padded_atoms(const Request *r, bool last) { return last ? r->nbr : (r->nbr + 7) / 8 * 8; }

// Pattern statistics of the union of `g` (in order), padding atoms included.
marnoldi::PatternStats group_stats(const std::vector<Request *> &g)
{
    marnoldi::PatternStats u;
    int64_t span = 0;
    for (size_t q = 0; q < g.size(); ++q) {
        const marnoldi::PatternStats &a = g[q]->stats;
        const int64_t n = padded_atoms(g[q], q + 1 == g.size()), pad = n - a.nbr;
        u.nbr += n;
        u.nnzb += a.nnzb + pad;   // one (diagonal) block per padding atom
        u.nc += a.nc;
        u.prow += a.prow;
        u.maxrow = std::max(u.maxrow, a.maxrow);
        span = std::max(span, n);
    }
    u.m_vec = 4 * span;
    return u;
}

bool groupable(const Request *a, const Request *b)
{
    // kT enters only each member's own Fermi step (marnoldi_set_member_temperatures)
    return a->region_atoms == 0 && b->region_atoms == 0 && a->prec == b->prec && a->nu == b->nu &&
           a->nu <= 253 && a->nu <= a->stats.nc && b->nu <= b->stats.nc &&
           a->m_pad == b->m_pad && (a->rho == nullptr) == (b->rho == nullptr);
}

// One request from setup to read-back on `stream`.
void run_request(marnoldi_server *srv, Request *r, cudaStream_t stream)
{
    marnoldi_ctx *ctx = nullptr;
    int rc = marnoldi::setup_with_allocator(&ctx, r->nbr, r->rp, r->ci, r->H, r->S, r->mask, r->pos,
                                            r->box, r->prec, (void *)stream, pool_alloc, pool_free, srv);
    if (rc) {
        r->status = rc;
        r->msg = marnoldi_last_error(nullptr);
        return;
    }
    rc = marnoldi_set_batch(ctx, r->batch);
    if (!rc) rc = marnoldi_solve(ctx, nullptr, -1, r->nu, r->region_atoms, r->electron_count, r->kT, nullptr);
    if (!rc && r->rho) rc = marnoldi_density(ctx, r->rho, r->rhoE);
    if (!rc) rc = marnoldi_energy(ctx, &r->E, &r->mu, &r->N);
    if (rc) r->msg = marnoldi_last_error(ctx);
    r->status = rc;
    marnoldi_destroy(ctx);
}

// Several requests as the members of one union, on `stream`; every member
// gets the union's status.
void run_group(marnoldi_server *srv, const std::vector<Request *> &g, int64_t batch, cudaStream_t stream)
{
    // the union: member q's atoms from off[q], its blocks from boff[q]; padding
    // atoms carry one block (H = 0, S = I) and four padding orbitals
    std::vector<int64_t> off(g.size() + 1, 0), boff(g.size(), 0), rp(1, 0);
    std::vector<int32_t> ci;
    std::vector<double> H, S, ne, kT;
    std::vector<uint8_t> mask;
    int64_t nb = 0;
    for (size_t q = 0; q < g.size(); ++q) {
        const Request *r = g[q];
        const int64_t n = padded_atoms(r, q + 1 == g.size()), nnzb = r->rp[r->nbr];
        boff[q] = nb;
        for (int64_t I = 1; I <= r->nbr; ++I) rp.push_back(nb + r->rp[I]);
        for (int64_t k = 0; k < nnzb; ++k) ci.push_back((int32_t)(r->ci[k] + off[q]));
        H.insert(H.end(), r->H, r->H + 16 * nnzb);
        S.insert(S.end(), r->S, r->S + 16 * nnzb);
        if (r->mask) mask.insert(mask.end(), r->mask, r->mask + 4 * r->nbr);
        else mask.insert(mask.end(), 4 * r->nbr, (uint8_t)1);
        nb += nnzb;
        for (int64_t p = r->nbr; p < n; ++p) {
            rp.push_back(++nb);
            ci.push_back((int32_t)(off[q] + p));
            for (int e = 0; e < 16; ++e) {
                H.push_back(0.0);
                S.push_back(e % 5 == 0 ? 1.0 : 0.0);
            }
            mask.insert(mask.end(), 4, (uint8_t)0);
        }
        off[q + 1] = off[q] + n;
        ne.push_back(r->electron_count);
        kT.push_back(r->kT);
    }
    const Request *r0 = g[0];
    auto finish = [&](int rc, const char *msg) {
        for (Request *r : g) {
            r->status = rc;
            if (rc) r->msg = msg;
        }
    };
    marnoldi_ctx *ctx = nullptr;
    int rc = marnoldi::setup_with_allocator(&ctx, off.back(), rp.data(), ci.data(), H.data(), S.data(),
                                            mask.data(), nullptr, nullptr, r0->prec, (void *)stream, pool_alloc,
                                            pool_free, srv);
    if (rc) {
        finish(rc, marnoldi_last_error(nullptr));
        return;
    }
    rc = marnoldi_set_members(ctx, (int)g.size(), off.data(), ne.data());
    if (!rc) rc = marnoldi_set_member_temperatures(ctx, (int)g.size(), kT.data());
    if (!rc) rc = marnoldi_set_batch(ctx, batch);
    if (!rc) rc = marnoldi_solve(ctx, nullptr, -1, r0->nu, 0, 0.0, r0->kT, nullptr);
    if (!rc && r0->rho) {
        std::vector<double> rho(16 * (size_t)nb), rhoE(16 * (size_t)nb);
        rc = marnoldi_density(ctx, rho.data(), rhoE.data());
        for (size_t q = 0; q < g.size() && !rc; ++q) {
            const size_t n16 = 16 * (size_t)g[q]->rp[g[q]->nbr];
            memcpy(g[q]->rho, rho.data() + 16 * boff[q], n16 * sizeof(double));
            memcpy(g[q]->rhoE, rhoE.data() + 16 * boff[q], n16 * sizeof(double));
        }
    }
    for (size_t q = 0; q < g.size() && !rc; ++q)
        rc = marnoldi_member_energy(ctx, (int)q, &g[q]->E, &g[q]->mu, &g[q]->N);
    finish(rc, rc ? marnoldi_last_error(ctx) : "");
    marnoldi_destroy(ctx);
}

void worker_main(marnoldi_server *srv, int w)
{
    cudaSetDevice(srv->device);
    const cudaStream_t stream = srv->streams[w];
    std::unique_lock<std::mutex> lock(srv->mu);
    for (;;) {
        // FIFO admission: the head of the queue starts when its footprint fits
        srv->cv_admit.wait(lock, [&] {
            return srv->stopping ||
                   (!srv->queue.empty() && srv->in_use + srv->queue.front()->bytes <= srv->budget);
        });
        if (srv->stopping) return;
        Request *r = srv->queue.front();
        srv->queue.pop_front();
        // continuous batching: queued requests that can share r's launches join
        // it while the union's footprint fits beside the running requests
        std::vector<Request *> g{r};
        size_t bytes = r->bytes;
        int64_t batch = r->batch;
        if (srv->max_group > 1) {
            int64_t atoms = padded_atoms(r, false);
            const size_t share = srv->budget / (size_t)srv->workers;
            for (auto it = srv->queue.begin(); it != srv->queue.end() && (int)g.size() < srv->max_group;) {
                Request *x = *it;
                if (!groupable(r, x) || atoms + x->nbr > kGroupAtoms) {
                    ++it;
                    continue;
                }
                g.push_back(x);
                size_t b = 0;
                int64_t used = 0;
                const int rc = choose_batch(group_stats(g), r->prec, r->nu, 0, nullptr, 0,
                                            std::max(share, bytes), &b, &used);
                if (rc || srv->in_use + b > srv->budget) {
                    g.pop_back();
                    break;
                }
                bytes = b;
                batch = used;
                atoms += padded_atoms(x, false);
                it = srv->queue.erase(it);
            }
        }
        srv->in_use += bytes;
        srv->peak = std::max(srv->peak, srv->in_use);
        ++srv->running;
        srv->peak_running = std::max(srv->peak_running, srv->running);
        if (g.size() > 1) {
            ++srv->groups;
            srv->largest_group = std::max<int64_t>(srv->largest_group, (int64_t)g.size());
        }
        const double t_start = srv->now();
        for (Request *x : g) {
            x->t_start = t_start;
            x->bytes = g.size() > 1 ? bytes : x->bytes;
            x->batch = g.size() > 1 ? batch : x->batch;
        }
        // the next head may fit beside this one
        srv->cv_admit.notify_all();
        lock.unlock();
        if (g.size() == 1) run_request(srv, r, stream);
        else run_group(srv, g, batch, stream);
        lock.lock();
        const double t_end = srv->now();
        for (Request *x : g) {
            x->t_end = t_end;
            x->done = true;
        }
        srv->in_use -= bytes;
        --srv->running;
        srv->completed += (int64_t)g.size();
        srv->cv_done.notify_all();
        srv->cv_admit.notify_all();
    }
}

}  // namespace

extern "C" {

int marnoldi_server_create(marnoldi_server **out, int workers, size_t hbm_budget_bytes)
{
    t_server_err.clear();
    if (!out) return server_fail(MARNOLDI_EINVAL, "out is NULL");
    *out = nullptr;
    if (workers < 1 || workers > 64) return server_fail(MARNOLDI_EINVAL, "workers must be in [1, 64]");
    if (hbm_budget_bytes < ((size_t)1 << 20)) return server_fail(MARNOLDI_EINVAL, "budget below 1 MiB");
    auto srv = std::make_unique<marnoldi_server>();
    srv->budget = hbm_budget_bytes;
    srv->workers = workers;
    srv->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&srv->device);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = srv->device;
    if (e == cudaSuccess) e = cudaMemPoolCreate(&srv->pool, &props);
    if (e == cudaSuccess) {
        // keep up to the budget mapped between requests; never make one
        // stream's allocation wait for another stream's free
        uint64_t keep = hbm_budget_bytes;
        int no = 0;
        e = cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e == cudaSuccess)
            e = cudaMemPoolSetAttribute(srv->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    for (int w = 0; w < workers && e == cudaSuccess; ++w) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) srv->streams.push_back(s);
    }
    if (e != cudaSuccess) {
        const std::string m = std::string("server setup: ") + cudaGetErrorString(e);
        cudaGetLastError();
        for (auto s : srv->streams) cudaStreamDestroy(s);
        if (srv->pool) cudaMemPoolDestroy(srv->pool);
        return server_fail(MARNOLDI_ECUDA, m.c_str());
    }
    marnoldi_server *p = srv.release();
    for (int w = 0; w < workers; ++w) p->threads.emplace_back(worker_main, p, w);
    *out = p;
    return MARNOLDI_OK;
}

int marnoldi_server_submit(marnoldi_server *srv, int64_t n_block_rows, const int64_t *row_ptr,
                           const int32_t *col_idx, const double *H_vals, const double *S_vals,
                           const uint8_t *orbital_mask, const double *positions, const double *box,
                           int precision, int nu, int region_atoms, double electron_count, double kT,
                           int64_t batch_columns, double *rho_vals, double *rhoE_vals,
                           int64_t *request_id)
{
    t_server_err.clear();
    if (!srv || !request_id) return server_fail(MARNOLDI_EINVAL, "server or request_id is NULL");
    *request_id = 0;
    if (!col_idx || !H_vals || !S_vals) return server_fail(MARNOLDI_EINVAL, "NULL matrix array");
    if ((rho_vals == nullptr) != (rhoE_vals == nullptr))
        return server_fail(MARNOLDI_EINVAL, "rho_vals and rhoE_vals must be given together");
    if (batch_columns < 0) return server_fail(MARNOLDI_EINVAL, "batch_columns must be >= 0");
    if (!(kT > 0.0) || !std::isfinite(kT) || !(electron_count > 0.0) || !std::isfinite(electron_count))
        return server_fail(MARNOLDI_EINVAL, "kT and electron_count must be positive and finite");
    auto r = std::make_unique<Request>();
    r->t_submit = srv->now();
    // batch size: the caller's, else the largest whose footprint stays within
    // budget / workers (footprints grow with the batch), at least one column
    size_t bytes = 0;
    int64_t used = 0;
    int rc = MARNOLDI_OK;
    if (n_block_rows < 1 || n_block_rows > (int64_t)1 << 30 || !row_ptr)
        return server_fail(MARNOLDI_EINVAL, "need n_block_rows >= 1 and row_ptr");
    if ((rc = marnoldi::pattern_stats(n_block_rows, row_ptr, orbital_mask, r->stats)) ||
        (rc = choose_batch(r->stats, precision, nu, region_atoms, box, batch_columns,
                           srv->budget / (size_t)srv->workers, &bytes, &used)))
        return server_fail(rc, marnoldi_last_error(nullptr));
    r->m_pad = marnoldi::column_shape(4 * n_block_rows, precision).m_pad;
    if (bytes > srv->budget) {
        char m[160];
        snprintf(m, sizeof m, "footprint %zu bytes exceeds the server budget of %zu bytes", bytes, srv->budget);
        return server_fail(MARNOLDI_ENOMEM, m);
    }
    r->nbr = n_block_rows;
    r->rp = row_ptr;
    r->ci = col_idx;
    r->H = H_vals;
    r->S = S_vals;
    r->mask = orbital_mask;
    r->pos = positions;
    r->box = box;
    r->prec = precision;
    r->nu = nu;
    r->region_atoms = region_atoms;
    r->electron_count = electron_count;
    r->kT = kT;
    r->rho = rho_vals;
    r->rhoE = rhoE_vals;
    r->batch = used;
    r->bytes = bytes;
    std::lock_guard<std::mutex> lock(srv->mu);
    if (srv->stopping) return server_fail(MARNOLDI_ESTATE, "server is shutting down");
    r->id = srv->next_id++;
    *request_id = r->id;
    srv->queue.push_back(r.get());
    srv->reqs.emplace(r->id, std::move(r));
    srv->cv_admit.notify_all();
    return MARNOLDI_OK;
}

int marnoldi_server_wait(marnoldi_server *srv, int64_t request_id, double timeout_s, int *status,
                         double *result, char *message, size_t message_cap)
{
    t_server_err.clear();
    if (!srv) return server_fail(MARNOLDI_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lock(srv->mu);
    auto it = srv->reqs.find(request_id);
    if (it == srv->reqs.end()) return server_fail(MARNOLDI_EINVAL, "unknown request id");
    Request *r = it->second.get();
    auto ready = [&] { return r->done; };
    if (timeout_s < 0.0) {
        srv->cv_done.wait(lock, ready);
    } else if (!srv->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), ready)) {
        return MARNOLDI_EPENDING;
    }
    if (result) {
        result[0] = r->E;
        result[1] = r->mu;
        result[2] = r->N;
        result[3] = r->t_submit;
        result[4] = r->t_start;
        result[5] = r->t_end;
        result[6] = (double)r->bytes;
        result[7] = (double)r->batch;
    }
    if (message && message_cap) {
        const size_t n = std::min(message_cap - 1, r->msg.size());
        memcpy(message, r->msg.data(), n);
        message[n] = '\0';
    }
    if (status) *status = r->status;
    srv->reqs.erase(it);
    return MARNOLDI_OK;
}

int marnoldi_server_stats(marnoldi_server *srv, int64_t *stats)
{
    if (!srv || !stats) return server_fail(MARNOLDI_EINVAL, "server or stats is NULL");
    std::lock_guard<std::mutex> lock(srv->mu);
    stats[0] = (int64_t)srv->queue.size();
    stats[1] = srv->running;
    stats[2] = srv->completed;
    stats[3] = (int64_t)srv->in_use;
    stats[4] = (int64_t)srv->peak;
    stats[5] = srv->peak_running;
    uint64_t reserved = 0;
    if (cudaMemPoolGetAttribute(srv->pool, cudaMemPoolAttrReservedMemHigh, &reserved) != cudaSuccess) {
        cudaGetLastError();
        reserved = 0;
    }
    stats[6] = (int64_t)reserved;
    stats[7] = srv->groups;
    stats[8] = srv->largest_group;
    return MARNOLDI_OK;
}

int marnoldi_server_set_group_limit(marnoldi_server *srv, int max_members)
{
    if (!srv || max_members < 1 || max_members > 64)
        return server_fail(MARNOLDI_EINVAL, "max_members must be in [1, 64]");
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->max_group = max_members;
    return MARNOLDI_OK;
}

const char *marnoldi_server_last_error(void) { return t_server_err.c_str(); }

void marnoldi_server_destroy(marnoldi_server *srv)
{
    if (!srv) return;
    {
        std::unique_lock<std::mutex> lock(srv->mu);
        // requests already queued still run; nothing new is accepted
        srv->cv_done.wait(lock, [&] { return srv->queue.empty() && srv->running == 0; });
        srv->stopping = true;
        srv->cv_admit.notify_all();
    }
    for (auto &t : srv->threads) t.join();
    for (auto s : srv->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    cudaMemPoolDestroy(srv->pool);
    cudaGetLastError();
    delete srv;
}

}  // extern "C"
