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
// Results do not depend on the mix: a request's kernels see only its own
// data, its batch size changes which columns share a launch but not any
// column's arithmetic, and its reductions run in a fixed order.
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
    int64_t next_id = 1, completed = 0;
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
        srv->in_use += r->bytes;
        srv->peak = std::max(srv->peak, srv->in_use);
        ++srv->running;
        srv->peak_running = std::max(srv->peak_running, srv->running);
        r->t_start = srv->now();
        // the next head may fit beside this one
        srv->cv_admit.notify_all();
        lock.unlock();
        run_request(srv, r, stream);
        lock.lock();
        r->t_end = srv->now();
        r->done = true;
        srv->in_use -= r->bytes;
        --srv->running;
        ++srv->completed;
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
    int rc;
    if (batch_columns > 0) {
        rc = marnoldi_footprint(n_block_rows, row_ptr, orbital_mask, box, precision, nu, region_atoms,
                                batch_columns, &bytes, &used);
    } else {
        rc = marnoldi_footprint(n_block_rows, row_ptr, orbital_mask, box, precision, nu, region_atoms,
                                (int64_t)1 << 40, &bytes, &used);   // every column in one batch
        const size_t share = srv->budget / (size_t)srv->workers;
        if (!rc && bytes > share) {
            int64_t lo = 1, hi = used;   // footprint(lo) may exceed the share; hi does
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo + 1) / 2;
                size_t b = 0;
                if ((rc = marnoldi_footprint(n_block_rows, row_ptr, orbital_mask, box, precision, nu,
                                             region_atoms, mid, &b, nullptr)))
                    break;
                if (b <= share) lo = mid; else hi = mid - 1;
            }
            if (!rc) rc = marnoldi_footprint(n_block_rows, row_ptr, orbital_mask, box, precision, nu,
                                             region_atoms, lo, &bytes, &used);
        }
    }
    if (rc) return server_fail(rc, marnoldi_last_error(nullptr));
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
