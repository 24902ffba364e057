// Serving engine: SpMV and CG-solve requests against a pool of
// device-resident ARG-CSR matrices, with continuous batching.
//
// One worker thread owns the GPU side.  Each pass of its loop
//   1. retires finished work (an event per in-flight job) and frees its
//      stream slot and memory;
//   2. advances every CG job whose last step has completed (a job is a
//      resumable state machine: a step is a few inner iterations; all solver
//      scalars stay on the device);
//   3. admits queued requests, oldest first, while a stream slot and HBM
//      budget are free: SpMV requests on the same matrix are fused, up to
//      max_batch of them, into one SpMM launch (their x vectors packed as
//      the columns of X); a CG request becomes a job on its own stream.
//      CG jobs never take the last spmv_streams slots, so SpMV requests
//      pass CG requests that wait for a slot or for memory.
// Work admitted while other requests run overlaps with them on the device.
// The paper has no serving layer; this is the library's runtime around its
// SpMV (Section 1 names iterative solvers as the consumer).
#include <math.h>

#include <chrono>
#include <condition_variable>
#include <atomic>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace argcsr {
namespace {

constexpr int kMaxBatch = 16;

double now_us() {
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

// x columns packed into X (n x k row-major) and Y unpacked into the y vectors.
struct PtrSet {
    const void *in[kMaxBatch];
    void *out[kMaxBatch];
};

template <typename T>
__global__ void k_pack(PtrSet p, int cnt, int k, long long n, T *__restrict__ X) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * k;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / k;
        const int j = (int)(i - r * k);
        X[i] = j < cnt ? static_cast<const T *>(p.in[j])[r] : T(0);
    }
}

template <typename T>
__global__ void k_unpack(PtrSet p, int cnt, int k, long long n, const T *__restrict__ Y) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * k;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / k;
        const int j = (int)(i - r * k);
        if (j < cnt) static_cast<T *>(p.out[j])[r] = Y[i];
    }
}

struct Request {
    int64_t id;
    int type;               // 0 SpMV, 1 CG
    int32_t matrix;
    const void *in;
    void *out;
    double tol;
    int32_t max_iters;
    argcsr_request_info info;
};

struct Matrix {
    argcsr_t A;
    argcsr_t Ares;
    size_t bytes;
};

struct Job {
    int stream;             // index into the stream pool
    size_t bytes;           // budget held
    std::vector<Request *> reqs;
    // SpMV batch
    cudaEvent_t ev = nullptr;
    void *X = nullptr, *Y = nullptr;
    // CG
    std::unique_ptr<CgJob> cg;
};

}  // namespace
}  // namespace argcsr

using namespace argcsr;

struct argcsr_server {
    argcsr_server_params P;
    int device;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    std::vector<Matrix> mats;
    std::atomic<size_t> matrix_bytes{0}, work_bytes{0};

    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Request *> pending;
    std::map<int64_t, std::unique_ptr<Request>> requests;
    int64_t next_id = 1;
    int64_t unfinished = 0;
    bool stop = false;
    std::thread worker;
    std::vector<std::unique_ptr<Job>> active;   // worker thread only
    int cg_running = 0;                         // worker thread only

    int free_stream() {
        for (size_t i = 0; i < streams.size(); ++i)
            if (!stream_busy[i]) return (int)i;
        return -1;
    }
    size_t budget_left() const {
        if (P.hbm_budget_bytes <= 0) return SIZE_MAX;
        const size_t cap = (size_t)P.hbm_budget_bytes;
        const size_t used = matrix_bytes + work_bytes;
        return used >= cap ? 0 : cap - used;
    }
    void finish(Request *r, argcsr_status st, double rel, int iters, int converged) {
        std::lock_guard<std::mutex> lock(mu);
        r->info.state = st == ARGCSR_OK ? 2 : 3;
        r->info.status = st;
        r->info.t_done_us = now_us();
        r->info.rel_residual = rel;
        r->info.iters = iters;
        r->info.converged = converged;
        --unfinished;
        done_cv.notify_all();
    }
    void release(Job &j) {
        stream_busy[j.stream] = false;
        if (j.reqs[0]->type == 1) --cg_running;
        work_bytes -= j.bytes;
        if (j.ev) cudaEventDestroy(j.ev);
        pool_free(j.X, streams[j.stream]);
        pool_free(j.Y, streams[j.stream]);
    }

    // SpMV requests on one matrix: a plain SpMV for one, an SpMM of the
    // packed x vectors for more.
    argcsr_status launch_spmv_batch(Job &j) {
        const Matrix &m = mats[j.reqs[0]->matrix];
        cudaStream_t s = streams[j.stream];
        const int cnt = (int)j.reqs.size();
        argcsr_status st = ARGCSR_OK;
        if (cnt == 1) {
            st = launch_spmv(m.A, j.reqs[0]->in, j.reqs[0]->out, s);
        } else {
            int k = 2;
            while (k < cnt) k <<= 1;
            const size_t es = vec_size(m.A->dtype);
            PtrSet ps{};
            for (int i = 0; i < cnt; ++i) { ps.in[i] = j.reqs[i]->in; ps.out[i] = j.reqs[i]->out; }
            if ((st = pool_alloc(&j.X, (size_t)m.A->n_cols * k * es, s)) != ARGCSR_OK) return st;
            if ((st = pool_alloc(&j.Y, (size_t)m.A->n_rows * k * es, s)) != ARGCSR_OK) return st;
            const long long nc = m.A->n_cols, nr = m.A->n_rows;
            const unsigned gp = (unsigned)min((nc * k + 255) / 256, 152LL * 16);
            const unsigned gu = (unsigned)min((nr * k + 255) / 256, 152LL * 16);
            if (es == 8) k_pack<double><<<max(gp, 1u), 256, 0, s>>>(ps, cnt, k, nc, (double *)j.X);
            else k_pack<float><<<max(gp, 1u), 256, 0, s>>>(ps, cnt, k, nc, (float *)j.X);
            st = launch_spmm_public(m.A, k, j.X, k, j.Y, k, s);
            if (st == ARGCSR_OK) {
                if (es == 8) k_unpack<double><<<max(gu, 1u), 256, 0, s>>>(ps, cnt, k, nr, (const double *)j.Y);
                else k_unpack<float><<<max(gu, 1u), 256, 0, s>>>(ps, cnt, k, nr, (const float *)j.Y);
                count_launches(2);
            }
        }
        if (st != ARGCSR_OK) return st;
        cudaError_t e = cudaEventCreateWithFlags(&j.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(j.ev, s);
        return e == cudaSuccess ? ARGCSR_OK : record_cuda(e, "server spmv batch");
    }

    size_t spmv_bytes(const Matrix &m, int cnt) const {
        if (cnt <= 1) return 0;
        int k = 2;
        while (k < cnt) k <<= 1;
        return ((size_t)m.A->n_cols + m.A->n_rows) * k * vec_size(m.A->dtype) + 512;
    }

    // Admit queued requests while a stream and memory are free.  Returns
    // false if nothing could be admitted.
    bool admit() {
        bool any = false;
        bool cg_blocked = false;
        for (;;) {
            if ((int)active.size() >= P.max_inflight) break;
            const int sidx = free_stream();
            if (sidx < 0) break;
            std::vector<Request *> take;
            size_t need = 0;
            {
                std::lock_guard<std::mutex> lock(mu);
                if (pending.empty()) break;
                // the oldest request that may start now: CG jobs leave
                // spmv_streams slots to SpMV batches, so short requests do
                // not queue behind long solves
                const bool cg_ok = !cg_blocked && cg_running < (int)streams.size() - P.spmv_streams;
                Request *head = nullptr;
                for (Request *r : pending)
                    if (r->type == 0 || cg_ok) { head = r; break; }
                if (!head) break;
                const Matrix &m = mats[head->matrix];
                if (head->type == 0) {
                    // the head and later SpMV requests on the same matrix
                    for (auto it = pending.begin(); it != pending.end() && (int)take.size() < P.max_batch; ++it)
                        if ((*it)->type == 0 && (*it)->matrix == head->matrix) take.push_back(*it);
                    while (!take.empty() && spmv_bytes(m, (int)take.size()) > budget_left()) take.pop_back();
                    if (take.empty()) take.push_back(head);   // k = 1 needs no memory
                    need = spmv_bytes(m, (int)take.size());
                } else {
                    need = cg_job_bytes(m.A);
                    if (need > budget_left()) {
                        if (active.empty() && work_bytes == 0) {
                            // it can never fit: fail it rather than wait forever
                            for (auto it = pending.begin(); it != pending.end(); ++it)
                                if (*it == head) { pending.erase(it); break; }
                            head->info.state = 3;
                            head->info.status = ARGCSR_ENOMEM;
                            head->info.t_done_us = now_us();
                            --unfinished;
                            done_cv.notify_all();
                            continue;
                        }
                        cg_blocked = true;   // wait for memory; SpMV may still go
                        continue;
                    }
                    take.push_back(head);
                }
                for (Request *r : take) {
                    for (auto it = pending.begin(); it != pending.end(); ++it)
                        if (*it == r) { pending.erase(it); break; }
                    r->info.state = 1;
                    r->info.t_start_us = now_us();
                    r->info.batch = (int32_t)take.size();
                }
            }
            auto job = std::make_unique<Job>();
            job->stream = sidx;
            job->bytes = need;
            job->reqs = take;
            stream_busy[sidx] = true;
            work_bytes += need;
            if (take[0]->type == 1) ++cg_running;
            argcsr_status st;
            if (take[0]->type == 0) {
                st = launch_spmv_batch(*job);
            } else {
                const Matrix &m = mats[take[0]->matrix];
                argcsr_cg_params cp{take[0]->tol, 0.0, take[0]->max_iters, 50, P.cg_check_every, 0};
                job->cg.reset(make_cg_job(m.A, m.Ares, static_cast<const double *>(take[0]->in),
                                          static_cast<double *>(take[0]->out), cp, streams[sidx]));
                st = job->cg ? job->cg->start() : ARGCSR_ENOMEM;
            }
            if (st != ARGCSR_OK) {
                for (Request *r : take) finish(r, st, 0.0, 0, 0);
                cudaStreamSynchronize(streams[sidx]);
                job->cg.reset();
                release(*job);
                continue;
            }
            active.push_back(std::move(job));
            any = true;
        }
        return any;
    }

    // Retire finished SpMV batches; advance or retire CG jobs.
    bool progress() {
        bool any = false;
        for (size_t i = 0; i < active.size();) {
            Job &j = *active[i];
            bool done = false;
            if (!j.cg) {
                cudaError_t e = cudaEventQuery(j.ev);
                if (e != cudaErrorNotReady) {
                    for (Request *r : j.reqs)
                        finish(r, e == cudaSuccess ? ARGCSR_OK : record_cuda(e, "server spmv"), 0.0, 0, 0);
                    done = true;
                }
            } else if (j.cg->step_done()) {
                argcsr_status st = j.cg->advance();
                if (st != ARGCSR_OK || j.cg->finished()) {
                    argcsr_cg_result res{};
                    j.cg->result(&res);
                    if (st == ARGCSR_OK) st = j.cg->status();
                    finish(j.reqs[0], st, res.rel_residual, res.inner_iters, res.converged);
                    done = true;
                }
            }
            if (done) {
                j.cg.reset();   // frees the job's workspace on its stream
                release(j);
                active.erase(active.begin() + i);
                any = true;
            } else {
                ++i;
            }
        }
        return any;
    }

    void loop() {
        cudaSetDevice(device);
        for (;;) {
            {
                std::unique_lock<std::mutex> lock(mu);
                if (stop && pending.empty() && active.empty()) return;
                if (active.empty() && pending.empty())
                    cv.wait_for(lock, std::chrono::milliseconds(50));
            }
            const bool moved = progress() | admit();
            if (!moved && !active.empty()) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
};

extern "C" {

ARGCSR_API argcsr_status argcsr_server_create(const argcsr_server_params *params, argcsr_server_t *out) {
    if (!out) return ARGCSR_EINVAL;
    *out = nullptr;
    argcsr_server_params P = params ? *params : argcsr_server_params{0, 0, 0, 0, 0, 0};
    if (P.hbm_budget_bytes < 0 || P.max_inflight < 0 || P.num_streams < 0 || P.max_batch < 0 ||
        P.max_batch > kMaxBatch || P.cg_check_every < 0 || P.spmv_streams < 0)
        return ARGCSR_EINVAL;
    if (P.max_inflight == 0) P.max_inflight = 64;
    if (P.num_streams == 0) P.num_streams = 8;
    if (P.spmv_streams >= P.num_streams) return ARGCSR_EINVAL;
    if (P.spmv_streams == 0) P.spmv_streams = P.num_streams >= 4 ? P.num_streams / 4 : P.num_streams - 1;
    if (P.max_batch == 0) P.max_batch = kMaxBatch;
    if (P.cg_check_every == 0) P.cg_check_every = 16;
    auto *S = new argcsr_server();
    S->P = P;
    cudaGetDevice(&S->device);
    for (int i = 0; i < P.num_streams; ++i) {
        cudaStream_t st;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t q : S->streams) cudaStreamDestroy(q);
            delete S;
            return record_cuda(e, "argcsr_server_create");
        }
        S->streams.push_back(st);
        S->stream_busy.push_back(false);
    }
    S->worker = std::thread([S] { S->loop(); });
    *out = S;
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_server_add_matrix(argcsr_server_t S, argcsr_t A, argcsr_t A_residual,
                                                  int32_t *id) {
    if (!S || !A || !id) return ARGCSR_EINVAL;
    if (A_residual && (A_residual->n_rows != A->n_rows || A_residual->n_cols != A->n_cols)) return ARGCSR_EINVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    const size_t bytes = (size_t)A->device_bytes + (A_residual && A_residual != A ? (size_t)A_residual->device_bytes : 0);
    if (S->P.hbm_budget_bytes > 0 && S->matrix_bytes + bytes > (size_t)S->P.hbm_budget_bytes) return ARGCSR_ENOMEM;
    if (S->next_id > 1) return ARGCSR_EINVAL;   // the pool is fixed once requests arrive
    S->mats.push_back({A, A_residual, bytes});
    S->matrix_bytes += bytes;
    *id = (int32_t)S->mats.size() - 1;
    return ARGCSR_OK;
}

static argcsr_status submit(argcsr_server_t S, int type, int32_t matrix, const void *in, void *out,
                            double tol, int32_t max_iters, int64_t *request) {
    if (!S || !request || !in || !out) return ARGCSR_EINVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop || matrix < 0 || matrix >= (int32_t)S->mats.size()) return ARGCSR_EINVAL;
    const Matrix &m = S->mats[matrix];
    if (type == 1 && (m.A->n_rows != m.A->n_cols || !(tol > 0))) return ARGCSR_EINVAL;
    auto r = std::make_unique<Request>();
    r->id = S->next_id++;
    r->type = type;
    r->matrix = matrix;
    r->in = in;
    r->out = out;
    r->tol = tol;
    r->max_iters = max_iters > 0 ? max_iters : 20000;
    r->info = argcsr_request_info{0, 0, 0, 0, 0, 0, now_us(), 0.0, 0.0, 0.0};
    *request = r->id;
    if (m.A->n_rows == 0) {
        // nothing to compute: done on arrival
        r->info.state = 2;
        r->info.converged = type == 1;
        r->info.t_start_us = r->info.t_done_us = r->info.t_submit_us;
        S->requests[r->id] = std::move(r);
        return ARGCSR_OK;
    }
    S->pending.push_back(r.get());
    S->requests[r->id] = std::move(r);
    ++S->unfinished;
    S->cv.notify_all();
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_server_submit_spmv(argcsr_server_t S, int32_t matrix, const void *d_x,
                                                   void *d_y, int64_t *request) {
    return submit(S, 0, matrix, d_x, d_y, 0.0, 0, request);
}

ARGCSR_API argcsr_status argcsr_server_submit_cg(argcsr_server_t S, int32_t matrix, const double *d_b,
                                                 double *d_x, double tol, int32_t max_iters,
                                                 int64_t *request) {
    return submit(S, 1, matrix, d_b, d_x, tol, max_iters, request);
}

ARGCSR_API argcsr_status argcsr_server_query(argcsr_server_t S, int64_t request, argcsr_request_info *info) {
    if (!S || !info) return ARGCSR_EINVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->requests.find(request);
    if (it == S->requests.end()) return ARGCSR_EINVAL;
    *info = it->second->info;
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_server_wait(argcsr_server_t S, int64_t request, double timeout_s,
                                            argcsr_request_info *info) {
    if (!S) return ARGCSR_EINVAL;
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->requests.find(request);
    if (it == S->requests.end()) return ARGCSR_EINVAL;
    Request *r = it->second.get();
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                              std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9));
    while (r->info.state < 2)
        if (S->done_cv.wait_until(lock, deadline) == std::cv_status::timeout) break;
    if (info) *info = r->info;
    return r->info.state >= 2 ? ARGCSR_OK : ARGCSR_ENOTSUP;
}

ARGCSR_API argcsr_status argcsr_server_release(argcsr_server_t S, int64_t request) {
    if (!S) return ARGCSR_EINVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->requests.find(request);
    if (it == S->requests.end() || it->second->info.state < 2) return ARGCSR_EINVAL;
    S->requests.erase(it);
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_server_drain(argcsr_server_t S, double timeout_s) {
    if (!S) return ARGCSR_EINVAL;
    std::unique_lock<std::mutex> lock(S->mu);
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                              std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9));
    while (S->unfinished > 0)
        if (S->done_cv.wait_until(lock, deadline) == std::cv_status::timeout) break;
    return S->unfinished == 0 ? ARGCSR_OK : ARGCSR_ENOTSUP;
}

ARGCSR_API argcsr_status argcsr_server_stats(argcsr_server_t S, int64_t *matrix_bytes, int64_t *work_bytes,
                                             int64_t *pending, int64_t *unfinished) {
    if (!S) return ARGCSR_EINVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    if (matrix_bytes) *matrix_bytes = (int64_t)S->matrix_bytes;
    if (work_bytes) *work_bytes = (int64_t)S->work_bytes;
    if (pending) *pending = (int64_t)S->pending.size();
    if (unfinished) *unfinished = S->unfinished;
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_server_destroy(argcsr_server_t S) {
    if (!S) return ARGCSR_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    S->worker.join();
    for (cudaStream_t s : S->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    delete S;
    return ARGCSR_OK;
}

}  // extern "C"
