// Serving loop: continuous batching of sampling jobs on one GPU.
//
// Jobs (one posterior each, with their own T and burn-in) are submitted from
// any host thread. A worker thread admits queued jobs in arrival order while
// their device footprint fits the HBM budget, steps all admitted jobs
// together (the batched engine of batch.cu: one tensor-core launch per layer
// over the rows of every active job), and between rounds of a few iterations
// retires the jobs that reached their T: final FP64 moments (MMSE and std) are
// copied to host memory, the job's device memory is freed and its completion
// time recorded. Jobs that arrive while others run join at the next round, so
// their work overlaps on the device. A job's chain does not depend on which
// other jobs share its steps.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "pnp_internal.h"

using namespace pnp;

namespace {

enum JobState { QUEUED = 0, RUNNING = 1, DONE = 2, FAILED = 3, CANCELLED = 4 };

struct ServerJob {
    int64_t id = 0;
    pnp_problem_desc desc;
    std::vector<float> y, h, x0;
    int T = 0, burn_in = 0;
    size_t footprint = 0;
    double t_submit = 0, t_admit = -1, t_done = -1;
    pnp_problem* p = nullptr;
    std::vector<double> mmse, sd;
    int state = QUEUED;
    pnp_status err = PNP_OK;
    std::string msg;
};

double now_s(const std::chrono::steady_clock::time_point& t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct pnp_server {
    const pnp_denoiser* D = nullptr;
    pnp_precision prec = PNP_BF16;
    size_t budget = 0, used = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int round_iters = 8;
    std::chrono::steady_clock::time_point t0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServerJob*> queue;
    std::map<int64_t, ServerJob*> jobs;
    std::vector<ServerJob*> active;
    BatchPlan plan;                                          // all active jobs
    std::map<std::vector<int64_t>, BatchPlan> subset_plans;  // rounds' smaller subsets
    int max_boost = 16;
    bool stop = false;
    int64_t next_id = 1;
    int64_t pixel_iters = 0;
    double device_s = 0.0;      // device time of the rounds' work (CUDA events)
};

// Device bytes a job needs: chain state, observation, kernel and denoiser scratch.
static size_t job_footprint(const pnp_problem_desc& d, const pnp_denoiser* D, pnp_precision prec) {
    const size_t N = (size_t)d.ny * d.nx, nc = (size_t)std::max(1, d.nchain);
    size_t b = N * 4 + (size_t)d.kh * d.kw * 4 + 5 * N * nc * 4 + 4096;
    if (d.noise_model == PNP_POISSON) b += 2 * N * nc * 4;   // z1, z2
    else b += N * 4;                                        // H^T y (one-pass or spectral gradient)
    if (d.noise_model == PNP_GAUSSIAN && !d.mask && is_wide(d.kh, d.kw) &&
        spectral_eligible(d.ny, d.nx, d.kh, d.kw))
        b += N * nc * 8 + N * 4 + (size_t)(d.ny + d.nx) * 8;   // spectra, |H^|^2, twiddles
    if (D) {
        b += prec == PNP_FP32 ? denoise_fp32_scratch(D->dev, d.ny, d.nx, (int)nc)
                              : denoise_bf16_scratch(D->dev, d.ny, d.nx, (int)nc);
    }
    return b;
}

static void retire(pnp_server* s, ServerJob* j) {
    // caller holds no lock; results are written before the state flips to DONE
    const size_t N = (size_t)j->desc.ny * j->desc.nx;
    j->mmse.assign(N, 0.0);
    j->sd.assign(N, 0.0);
    pnp_status st = pnp_get_moments(j->p, 0, j->mmse.data(), j->sd.data(), nullptr, 0);
    pnp_destroy_problem(j->p);
    j->p = nullptr;
    std::lock_guard<std::mutex> g(s->mu);
    j->t_done = now_s(s->t0);
    j->err = st;
    j->state = st == PNP_OK ? DONE : FAILED;
    if (st != PNP_OK) j->msg = pnp_last_error();
    s->used -= j->footprint;
    s->cv_done.notify_all();
}

static void worker_loop(pnp_server* s) {
    cudaSetDevice(s->device);
    bool changed = true;
    // events around each round's device work (admission copies and retirement
    // read-backs fall outside them)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    while (true) {
        std::vector<ServerJob*> admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty() || !s->active.empty(); });
            if (s->stop) break;
            // admission in arrival order while the footprint fits the budget
            while (!s->queue.empty()) {
                ServerJob* j = s->queue.front();
                if (j->state == CANCELLED) {
                    s->queue.pop_front();
                    continue;
                }
                if (s->used + j->footprint > s->budget) break;
                s->queue.pop_front();
                s->used += j->footprint;
                j->state = RUNNING;
                j->t_admit = now_s(s->t0);
                admit.push_back(j);
            }
        }
        for (ServerJob* j : admit) {
            pnp_problem_desc d = j->desc;
            d.stream = s->stream;
            pnp_status st = pnp_create_problem(&d, &j->p);
            if (st != PNP_OK) {
                std::lock_guard<std::mutex> g(s->mu);
                j->state = FAILED;
                j->err = st;
                j->msg = pnp_last_error();
                j->t_done = now_s(s->t0);
                s->used -= j->footprint;
                s->cv_done.notify_all();
                continue;
            }
            s->active.push_back(j);
            changed = true;
        }
        // drop jobs cancelled while running
        for (size_t k = 0; k < s->active.size();) {
            ServerJob* j = s->active[k];
            if (j->state == CANCELLED) {
                cudaStreamSynchronize(s->stream);
                pnp_destroy_problem(j->p);
                j->p = nullptr;
                {
                    std::lock_guard<std::mutex> g(s->mu);
                    s->used -= j->footprint;
                    j->t_done = now_s(s->t0);
                    s->cv_done.notify_all();
                }
                s->active.erase(s->active.begin() + k);
                changed = true;
            } else {
                ++k;
            }
        }
        if (s->active.empty()) continue;
        std::vector<pnp_problem*> probs;
        for (ServerJob* j : s->active) probs.push_back(j->p);
        if (changed) {
            for (auto& kv : s->subset_plans) plan_free(kv.second);
            s->subset_plans.clear();
            pnp_status st = plan_build(s->plan, probs, s->stream);
            if (st != PNP_OK) {
                // fail every active job; the server keeps serving new ones
                for (ServerJob* j : s->active) {
                    pnp_destroy_problem(j->p);
                    j->p = nullptr;
                    std::lock_guard<std::mutex> g(s->mu);
                    j->state = FAILED;
                    j->err = st;
                    j->t_done = now_s(s->t0);
                    s->used -= j->footprint;
                }
                s->active.clear();
                s->cv_done.notify_all();
                continue;
            }
            changed = false;
        }
        // a round, pixel-fair: every job gets round_iters iterations scaled by
        // (largest active job's pixels / its pixels), at most max_boost times more,
        // and never past its T. Small jobs thus finish early while large ones keep
        // the batch full; iteration i of the round steps the jobs with k_j > i.
        std::vector<int64_t> kj(s->active.size());
        int64_t pxmax = 1, kmax = 0;
        for (ServerJob* j : s->active)
            pxmax = std::max<int64_t>(pxmax, (int64_t)j->desc.ny * j->desc.nx * std::max(1, j->desc.nchain));
        for (size_t q = 0; q < s->active.size(); ++q) {
            ServerJob* j = s->active[q];
            const int64_t px = (int64_t)j->desc.ny * j->desc.nx * std::max(1, j->desc.nchain);
            int64_t k = s->round_iters * std::min<int64_t>(s->max_boost, std::max<int64_t>(1, pxmax / px));
            k = std::max<int64_t>(1, std::min<int64_t>(k, j->T - j->p->t));
            kj[q] = k;
            kmax = std::max(kmax, k);
        }
        pnp_status st = PNP_OK;
        std::vector<int64_t> prev_key;
        const BatchPlan* cur = nullptr;
        std::vector<pnp_problem*> sub;
        const bool timed = ev0 && ev1 && cudaEventRecord(ev0, s->stream) == cudaSuccess;
        for (int64_t i = 0; i < kmax && st == PNP_OK; ++i) {
            std::vector<int64_t> key;
            std::vector<pnp_problem*> members;
            for (size_t q = 0; q < s->active.size(); ++q)
                if (kj[q] > i) {
                    key.push_back(s->active[q]->id);
                    members.push_back(s->active[q]->p);
                }
            if (key != prev_key) {
                if (key.size() == s->active.size()) {
                    cur = &s->plan;
                } else {
                    auto it = s->subset_plans.find(key);
                    if (it == s->subset_plans.end()) {
                        it = s->subset_plans.emplace(key, BatchPlan()).first;
                        st = plan_build(it->second, members, s->stream);
                    }
                    cur = &it->second;
                }
                prev_key = key;
                sub = members;
            }
            if (st == PNP_OK) st = plan_enqueue_step(*cur, sub, s->stream);
        }
        if (timed) cudaEventRecord(ev1, s->stream);
        cudaError_t e = cudaStreamSynchronize(s->stream);
        float round_ms = 0.f;
        if (timed && e == cudaSuccess && cudaEventElapsedTime(&round_ms, ev0, ev1) != cudaSuccess)
            round_ms = 0.f;
        // a tensor-core layer whose bounded wait ran out (flags of the round's
        // jobs; the shared layers report into the first job's) fails the round
        for (size_t q = 0; q < s->active.size() && st == PNP_OK && e == cudaSuccess; ++q)
            st = take_timeout(s->active[q]->p->err, s->stream, "pnp_server");
        int64_t pix = 0;
        for (size_t q = 0; q < s->active.size(); ++q) {
            ServerJob* j = s->active[q];
            j->p->t += kj[q];
            pix += (int64_t)j->desc.ny * j->desc.nx * std::max(1, j->desc.nchain) * kj[q];
        }
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->pixel_iters += pix;
            s->device_s += 1e-3 * round_ms;
        }
        if (st != PNP_OK || e != cudaSuccess) {
            for (ServerJob* j : s->active) {
                pnp_destroy_problem(j->p);
                j->p = nullptr;
                std::lock_guard<std::mutex> g(s->mu);
                j->state = FAILED;
                j->err = st != PNP_OK ? st : PNP_ECUDA;
                j->t_done = now_s(s->t0);
                s->used -= j->footprint;
            }
            s->active.clear();
            s->cv_done.notify_all();
            changed = true;
            continue;
        }
        for (size_t q = 0; q < s->active.size();) {
            ServerJob* j = s->active[q];
            if (j->p->t >= j->T) {
                retire(s, j);
                s->active.erase(s->active.begin() + q);
                changed = true;
            } else {
                ++q;
            }
        }
    }
    // shutdown: release whatever is still on the device
    cudaStreamSynchronize(s->stream);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (ServerJob* j : s->active) {
        pnp_destroy_problem(j->p);
        j->p = nullptr;
    }
    s->active.clear();
}

extern "C" pnp_status pnp_server_create(const pnp_denoiser* D, pnp_precision prec,
                                        size_t hbm_budget_bytes, void* stream, pnp_server** out) {
    if (!out || hbm_budget_bytes == 0) return fail(PNP_EINVAL, "pnp_server_create: bad arguments");
    if (prec != PNP_FP32 && prec != PNP_BF16)
        return fail(PNP_ENOTSUP, "the server runs FP32 or BF16 denoisers");
    if (D && prec == PNP_BF16 && D->dev.F != 64) return fail(PNP_EINVAL, "BF16 serving needs F = 64");
    pnp_server* s = new pnp_server();
    s->D = D;
    s->prec = prec;
    s->budget = hbm_budget_bytes;
    s->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&s->device);
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete s;
            return cuda_fail(e, "cudaStreamCreate");
        }
        s->own_stream = true;
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return PNP_OK;
}

extern "C" pnp_status pnp_server_submit(pnp_server* s, const pnp_problem_desc* desc, int T,
                                        int burn_in, int64_t* job_id) {
    if (!s || !desc || !job_id || T < 1 || burn_in < 0)
        return fail(PNP_EINVAL, "pnp_server_submit: bad arguments");
    const pnp_problem_desc& d = *desc;
    if (d.ny < 1 || d.nx < 1 || !d.y || !d.h || d.kh < 1 || d.kw < 1)
        return fail(PNP_EINVAL, "pnp_server_submit: bad image or kernel");
    if (d.halo != 0) return fail(PNP_EINVAL, "pnp_server_submit: served jobs use halo = 0");
    ServerJob* j = new ServerJob();
    j->desc = d;
    j->desc.D = s->D;
    j->desc.precision = s->prec;
    j->desc.burn_in = burn_in;
    const size_t N = (size_t)d.ny * d.nx, nc = (size_t)std::max(1, d.nchain);
    j->y.assign(d.y, d.y + N);
    j->h.assign(d.h, d.h + (size_t)d.kh * d.kw);
    j->desc.y = j->y.data();
    j->desc.h = j->h.data();
    if (d.x0) {
        j->x0.assign(d.x0, d.x0 + N * nc);
        j->desc.x0 = j->x0.data();
    }
    j->T = T;
    j->burn_in = burn_in;
    j->footprint = job_footprint(j->desc, s->D, s->prec);
    if (j->footprint > s->budget) {
        const size_t fp = j->footprint;
        delete j;
        return fail(PNP_EBUSY, "job needs " + std::to_string(fp) + " device bytes, more than the budget " +
                                   std::to_string(s->budget));
    }
    std::lock_guard<std::mutex> g(s->mu);
    j->id = s->next_id++;
    j->t_submit = now_s(s->t0);
    s->jobs[j->id] = j;
    s->queue.push_back(j);
    *job_id = j->id;
    s->cv_work.notify_one();
    return PNP_OK;
}

extern "C" pnp_status pnp_server_poll(pnp_server* s, int64_t job_id, double* mmse, double* std,
                                      int* state) {
    if (!s || !state) return fail(PNP_EINVAL, "pnp_server_poll: bad arguments");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(PNP_EINVAL, "unknown job id");
    ServerJob* j = it->second;
    *state = j->state;
    if (j->state == FAILED) return fail(j->err, "job failed: " + j->msg);
    if (j->state == DONE) {
        if (mmse) memcpy(mmse, j->mmse.data(), j->mmse.size() * sizeof(double));
        if (std) memcpy(std, j->sd.data(), j->sd.size() * sizeof(double));
    }
    return PNP_OK;
}

extern "C" pnp_status pnp_server_wait(pnp_server* s, int64_t job_id, double timeout_s, int* state) {
    if (!s || !state) return fail(PNP_EINVAL, "pnp_server_wait: bad arguments");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(PNP_EINVAL, "unknown job id");
    ServerJob* j = it->second;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
        return j->state == DONE || j->state == FAILED || j->state == CANCELLED;
    });
    *state = j->state;
    if (!ok) return fail(PNP_ETIMEOUT, "job not finished within the timeout");
    return PNP_OK;
}

extern "C" pnp_status pnp_server_cancel(pnp_server* s, int64_t job_id) {
    if (!s) return fail(PNP_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(PNP_EINVAL, "unknown job id");
    ServerJob* j = it->second;
    if (j->state == QUEUED) {
        j->state = CANCELLED;
        j->t_done = now_s(s->t0);
        s->cv_done.notify_all();
    } else if (j->state == RUNNING) {
        j->state = CANCELLED;   // the worker frees it before its next round
    } else {
        return fail(PNP_ESTATE, "job already finished");
    }
    s->cv_work.notify_one();
    return PNP_OK;
}

extern "C" pnp_status pnp_server_job_times(pnp_server* s, int64_t job_id, double* t_submit,
                                           double* t_admit, double* t_done) {
    if (!s) return fail(PNP_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(PNP_EINVAL, "unknown job id");
    if (t_submit) *t_submit = it->second->t_submit;
    if (t_admit) *t_admit = it->second->t_admit;
    if (t_done) *t_done = it->second->t_done;
    return PNP_OK;
}

extern "C" pnp_status pnp_server_stats(pnp_server* s, int64_t* pixel_iters, int* active,
                                       int* queued, size_t* used_bytes) {
    if (!s) return fail(PNP_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    if (pixel_iters) *pixel_iters = s->pixel_iters;
    if (active) *active = (int)s->active.size();
    if (queued) *queued = (int)s->queue.size();
    if (used_bytes) *used_bytes = s->used;
    return PNP_OK;
}

extern "C" pnp_status pnp_server_device_seconds(pnp_server* s, double* seconds) {
    if (!s || !seconds) return fail(PNP_EINVAL, "pnp_server_device_seconds: bad arguments");
    std::lock_guard<std::mutex> g(s->mu);
    *seconds = s->device_s;
    return PNP_OK;
}

extern "C" pnp_status pnp_server_set_round(pnp_server* s, int iters, int max_boost) {
    if (!s || iters < 1 || max_boost < 1) return fail(PNP_EINVAL, "pnp_server_set_round: bad arguments");
    std::lock_guard<std::mutex> g(s->mu);
    s->round_iters = iters;
    s->max_boost = max_boost;
    return PNP_OK;
}

extern "C" void pnp_server_destroy(pnp_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    plan_free(s->plan);
    for (auto& kv : s->subset_plans) plan_free(kv.second);
    for (auto& kv : s->jobs) delete kv.second;
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}
