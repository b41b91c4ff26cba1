// Batched sampling: many independent posteriors (jobs) of different image
// sizes stepped together. One iteration of the batch runs, for every job that
// needs it, r = H x - y; then ONE first-layer launch over every job's state (a
// by-value job table), ONE tensor-core launch per F -> F layer and one for the
// last layer over the rows of all jobs (a device table of per-job tensor maps,
// balanced across the SMs to within a row), then every job's fused Langevin
// update. The whole iteration is captured once as a CUDA
// graph and replayed. Jobs never interact: each one's result is the same as
// when it runs alone (same kernels, same per-pixel summation order, its own
// Philox stream and step counter).
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "pnp_internal.h"

namespace pnp {

size_t BatchPlan::table_bytes(int n) { return (size_t)3 * n * sizeof(TcJob); }

// Activation planes of a BF16 problem (layout of denoise_bf16's scratch) and
// its timeout flag.
static void bf16_planes(const pnp_problem* p, __nv_bfloat16** A, __nv_bfloat16** B, int** err) {
    const size_t act = (size_t)p->nchain * p->ny * bf16_pad_width(p->nx) * 64;
    *A = (__nv_bfloat16*)p->scratch;
    *B = *A + act;
    *err = p->err;
}

pnp_status plan_build(BatchPlan& plan, const std::vector<pnp_problem*>& jobs, cudaStream_t s) {
    plan.n = (int)jobs.size();
    plan.total_rows = 0;
    if (plan.n == 0) return PNP_OK;
    const pnp_problem* p0 = jobs[0];
    plan.bf16 = p0->prec == PNP_BF16 && p0->D && p0->alpha != 0.0;
    if (!plan.bf16) return PNP_OK;
    const int K = p0->D->dev.K;
    const size_t need = BatchPlan::table_bytes(plan.n);
    if (plan.cap < need) {
        if (plan.tables) cudaFree(plan.tables);
        plan.tables = nullptr;
        plan.cap = 0;
        PNP_CUDA_TRY(cudaMalloc((void**)&plan.tables, need));
        plan.cap = need;
    }
    std::vector<TcJob> host(3 * (size_t)plan.n);
    int64_t row = 0;
    for (int j = 0; j < plan.n; ++j) {
        const pnp_problem* p = jobs[j];
        __nv_bfloat16 *A, *B;
        int* err;
        bf16_planes(p, &A, &B, &err);
        if (j == 0) plan.err = err;
        TcJob* ab = &host[j];
        TcJob* ba = &host[plan.n + j];
        TcJob* last = &host[2 * (size_t)plan.n + j];
        PNP_CUDA_TRY(tc_make_job(ab, A, B, p->ny, p->nx, p->nchain, nullptr, row));
        PNP_CUDA_TRY(tc_make_job(ba, B, A, p->ny, p->nx, p->nchain, nullptr, row));
        // after K-2 F -> F layers starting in A the activations are in B if K-2 is odd
        __nv_bfloat16* fin = ((K - 2) % 2 == 1) ? B : A;
        PNP_CUDA_TRY(tc_make_job(last, fin, nullptr, p->ny, p->nx, p->nchain, nullptr, row));
        last->xin = nullptr;   // the chain's update takes the residual G = x - D(x)
        last->dout = p->d;
        row += ab->rows;
    }
    plan.total_rows = row;
    PNP_CUDA_TRY(cudaMemcpyAsync(plan.tables, host.data(), need, cudaMemcpyHostToDevice, s));
    PNP_CUDA_TRY(cudaStreamSynchronize(s));
    return PNP_OK;
}

void plan_free(BatchPlan& plan) {
    if (plan.tables) cudaFree(plan.tables);
    plan.tables = nullptr;
    plan.cap = 0;
}

// r = H x - y for every job that forms it: one grouped launch per (kernel
// width, form) over the jobs with small kernels; wide kernels per job.
static pnp_status enqueue_residuals(const std::vector<pnp_problem*>& jobs, cudaStream_t s) {
    std::map<std::pair<int, bool>, std::vector<BlurArgs>> groups;
    for (pnp_problem* p : jobs) {
        if (p->inpaint || p->poisson || p->fused) continue;   // no residual plane this iteration
        if (is_wide(p->kh, p->kw)) {
            PNP_TRY(problem_pre(p, s));
            continue;
        }
        BlurArgs a{p->x, p->y, p->hsep ? p->hsep : p->h, p->kh, p->ny, p->nx, p->nchain,
                   1.0f, 0, p->r, 1.0f, 0};
        groups[{p->kw, p->hsep != nullptr}].push_back(a);
    }
    for (auto& g : groups)
        PNP_CUDA_TRY(launch_blur_group(g.second.data(), (int)g.second.size(), g.first.first,
                                       g.first.second, s));
    return PNP_OK;
}

// The x-updates (and Poisson z-updates) of every job: one grouped launch per
// (stencil width, form); inpainting and wide-kernel jobs per job. Every job's
// state buffer advances afterwards.
static pnp_status enqueue_updates(const std::vector<pnp_problem*>& jobs, cudaStream_t s) {
    std::map<std::pair<int, bool>, std::vector<UpdateParams>> ug;
    std::map<std::pair<int, bool>, std::vector<ZParams>> zg;
    std::vector<pnp_problem*> grouped;
    for (pnp_problem* p : jobs) {
        if (p->inpaint || is_wide(p->kh, p->kw)) {
            PNP_TRY(problem_post(p, s));   // advances its own state buffer
            continue;
        }
        UpdateParams u;
        PNP_TRY(problem_update_params(p, u));
        ug[{u.kw, u.hsep != nullptr}].push_back(u);
        if (p->poisson) {
            const ZParams z = problem_z_params(p);
            zg[{z.kw, z.hsep != nullptr}].push_back(z);
        }
        grouped.push_back(p);
    }
    for (auto& g : ug) PNP_CUDA_TRY(launch_update_group(g.second.data(), (int)g.second.size(), s));
    for (auto& g : zg) PNP_CUDA_TRY(launch_zupdate_group(g.second.data(), (int)g.second.size(), s));
    for (pnp_problem* p : grouped) problem_flip(p);
    return PNP_OK;
}

pnp_status plan_enqueue_step(const BatchPlan& plan, const std::vector<pnp_problem*>& jobs,
                             cudaStream_t s) {
    if (jobs.empty()) return PNP_OK;
    PNP_TRY(enqueue_residuals(jobs, s));
    const pnp_problem* p0 = jobs[0];
    if (p0->D && p0->alpha != 0.0) {
        const DenoiserDev& D = p0->D->dev;
        if (plan.bf16) {
            // the first layer of every job in one launch (each job's current state)
            std::vector<FirstJob> fj(jobs.size());
            for (size_t k = 0; k < jobs.size(); ++k) {
                const pnp_problem* p = jobs[k];
                __nv_bfloat16 *A, *B;
                int* err;
                bf16_planes(p, &A, &B, &err);
                memset(&fj[k], 0, sizeof(FirstJob));
                fj[k].x = p->x;
                fj[k].out = A;
                fj[k].ny = p->ny;
                fj[k].nx = p->nx;
                fj[k].nimg = p->nchain;
            }
            PNP_CUDA_TRY(first_layer_bf16_jobs(D, fj.data(), (int)fj.size(), plan.err, s));
            TcJob dummy;
            memset(&dummy, 0, sizeof(dummy));
            for (int k = 1; k < D.K - 1; ++k) {
                const TcJob* tab = plan.tables + ((k % 2 == 1) ? 0 : plan.n);   // A->B, B->A, ...
                PNP_CUDA_TRY(tc_launch(dummy, tab, plan.n, plan.total_rows,
                                       D.wtc + (size_t)(k - 1) * (3 * 8 * 192 * 8), D.hb + 64 * k,
                                       plan.err, false, s, false, nullptr, 1.f));
            }
            PNP_CUDA_TRY(tc_launch(dummy, plan.tables + 2 * (size_t)plan.n, plan.n, plan.total_rows,
                                   D.wtc_last, &D.last_bias, plan.err, true, s, false, nullptr, 1.f));
        } else {
            for (pnp_problem* p : jobs)
                PNP_CUDA_TRY(denoise_fp32(D, p->x, p->ny, p->nx, p->nchain, nullptr, p->d,
                                          (float*)p->scratch, s));
        }
    }
    return enqueue_updates(jobs, s);
}

}  // namespace pnp

using namespace pnp;

struct pnp_batch {
    std::vector<pnp_problem*> jobs;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    BatchPlan plan;
    // one graph per phase: every job steps each iteration, so the jobs' state
    // buffers alternate together (phase = iterations since creation mod 2)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::vector<int> graph_par[2];   // every job's state buffer when graph[k] was captured
    int phase = 0;
    bool eager_done = false;
};

extern "C" void pnp_batch_destroy(pnp_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (int k = 0; k < 2; ++k)
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    for (pnp_problem* p : b->jobs) pnp_destroy_problem(p);
    plan_free(b->plan);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

extern "C" pnp_status pnp_batch_create(const pnp_problem_desc* descs, int njobs, void* stream,
                                       pnp_batch** out) {
    if (!out || !descs || njobs < 1) return fail(PNP_EINVAL, "pnp_batch_create: bad arguments");
    *out = nullptr;
    const pnp_denoiser* D = descs[0].D;
    const pnp_precision prec = descs[0].precision;
    for (int j = 0; j < njobs; ++j) {
        if (descs[j].D != D || descs[j].precision != prec)
            return fail(PNP_EINVAL, "pnp_batch_create: all jobs must share the denoiser and precision");
        if (descs[j].halo != 0)
            return fail(PNP_EINVAL, "pnp_batch_create: batched jobs use the direct layout (halo = 0)");
        if (descs[j].precision != PNP_FP32 && descs[j].precision != PNP_BF16)
            return fail(PNP_ENOTSUP, "pnp_batch_create: batches run FP32 or BF16 denoisers");
    }
    pnp_batch* b = new pnp_batch();
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return cuda_fail(e, "cudaStreamCreate");
        }
        b->own_stream = true;
    }
    for (int j = 0; j < njobs; ++j) {
        pnp_problem_desc d = descs[j];
        d.stream = b->stream;
        pnp_problem* p = nullptr;
        pnp_status st = pnp_create_problem(&d, &p);
        if (st != PNP_OK) {
            const std::string msg = pnp_last_error();
            pnp_batch_destroy(b);
            return fail(st, "job " + std::to_string(j) + ": " + msg);
        }
        b->jobs.push_back(p);
    }
    pnp_status st = plan_build(b->plan, b->jobs, b->stream);
    if (st != PNP_OK) {
        pnp_batch_destroy(b);
        return st;
    }
    *out = b;
    return PNP_OK;
}

extern "C" pnp_status pnp_batch_step(pnp_batch* b, int n_iters) {
    if (!b || n_iters < 0) return fail(PNP_EINVAL, "pnp_batch_step: bad arguments");
    for (int i = 0; i < n_iters; ++i) {
        if (!b->eager_done || timer_enabled()) {
            // first iteration eagerly: performs the kernels' one-time setup outside capture
            PNP_TRY(plan_enqueue_step(b->plan, b->jobs, b->stream));
            b->eager_done = true;
        } else {
            cudaGraphExec_t& ge = b->graph[b->phase];
            std::vector<int> par0;
            for (pnp_problem* p : b->jobs) par0.push_back(p->par);
            if (ge && b->graph_par[b->phase] != par0) {
                // a job was stepped outside the batch: its buffers changed roles
                cudaGraphExecDestroy(ge);
                ge = nullptr;
            }
            if (!ge) {
                // capturing executes nothing: the jobs' state buffers are restored
                cudaGraph_t g = nullptr;
                PNP_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                pnp_status st = plan_enqueue_step(b->plan, b->jobs, b->stream);
                cudaError_t e = cudaStreamEndCapture(b->stream, &g);
                for (size_t k = 0; k < b->jobs.size(); ++k) {
                    b->jobs[k]->par = par0[k];
                    b->jobs[k]->x = b->jobs[k]->xb[par0[k]];
                }
                if (st != PNP_OK) {
                    if (g) cudaGraphDestroy(g);
                    return st;
                }
                if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) {
                    ge = nullptr;
                    return cuda_fail(e, "cudaGraphInstantiate");
                }
                b->graph_par[b->phase] = par0;
            }
            PNP_CUDA_TRY(cudaGraphLaunch(ge, b->stream));
            for (pnp_problem* p : b->jobs) problem_flip(p);
        }
        b->phase ^= 1;
        for (pnp_problem* p : b->jobs) p->t += 1;
    }
    return PNP_OK;
}

extern "C" pnp_status pnp_batch_sync(pnp_batch* b) {
    if (!b) return fail(PNP_EINVAL, "batch is NULL");
    PNP_CUDA_TRY(cudaStreamSynchronize(b->stream));
    // the layers shared by all jobs report into the first job's flag
    pnp_status st = PNP_OK;
    for (pnp_problem* p : b->jobs) {
        pnp_status sj = take_timeout(p->err, b->stream, "pnp_batch_sync");
        if (st == PNP_OK) st = sj;
    }
    return st;
}

extern "C" pnp_status pnp_batch_run(pnp_batch* b, int T, int burn_in) {
    if (!b || T < 0 || burn_in < 0) return fail(PNP_EINVAL, "pnp_batch_run: bad arguments");
    for (pnp_problem* p : b->jobs) {
        if (p->burn_in != burn_in) {
            p->burn_in = burn_in;
            PNP_CUDA_TRY(cudaMemcpyAsync(&p->st->burn_in, &burn_in, 4, cudaMemcpyHostToDevice, b->stream));
            PNP_CUDA_TRY(cudaStreamSynchronize(b->stream));
        }
    }
    PNP_TRY(pnp_batch_step(b, T));
    return pnp_batch_sync(b);
}

extern "C" pnp_status pnp_batch_job(pnp_batch* b, int job, pnp_problem** p) {
    if (!b || !p || job < 0 || job >= (int)b->jobs.size())
        return fail(PNP_EINVAL, "pnp_batch_job: bad arguments");
    *p = b->jobs[job];
    return PNP_OK;
}

extern "C" int pnp_batch_size(const pnp_batch* b) { return b ? (int)b->jobs.size() : 0; }
