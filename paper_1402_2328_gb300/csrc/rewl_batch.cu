// rewl_batch.cu -- many independent REWL instances (uneven lattice size, model, window count,
// walkers per window) advanced together: one move-kernel launch over a job grid (each CTA
// serves up to `walkers_per_block` walkers of one instance), then batched flatness/advance,
// exchange and round-end kernels driven by index tables; rounds are captured in CUDA graphs.
// Every instance evolves exactly as it would alone (its own seed, instance id and state).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "rewl.h"
#include "rewl_device.cuh"
#include "rewl_handle.h"
#include "rewl_kernels.cuh"

using namespace rewl;

struct rewl_batch_s {
    std::vector<rewl_t> inst;
    long long interval = 10000;
    int wpb = 0; // 0: automatic
    int thread_sites = 0; // instances with at most this many sites run one thread per walker
    int graph_rounds = 32, check_all = 0, profile = 0;
    bool inited = false;
    cudaStream_t stream = nullptr;
    // device tables
    State *d_states = nullptr;
    int4 *d_jobs = nullptr;
    int2 *d_chk = nullptr, *d_swp = nullptr;
    double2 *d_prm = nullptr;
    int njobs = 0, nchk = 0, nswp = 0, block_walkers = 1, wpb_used = 4;
    size_t smem = 0;
    std::vector<DevStatus> hst;
    DevStatus *h_status = nullptr; // pinned, one per instance
    cudaGraphExec_t graph = nullptr;
    int graph_len = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used, ev_free;
    std::string err;
    double seconds = 0.0;
    int sms = 148;

    int fail(int code, const std::string &m)
    {
        err = m;
        g_err = m;
        return code;
    }
    int cuda_fail(cudaError_t e, const char *where)
    {
        return fail(REWL_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    }
};

static void free_tables(rewl_batch_t b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    cudaFree(b->d_states);
    cudaFree(b->d_jobs);
    cudaFree(b->d_chk);
    cudaFree(b->d_swp);
    cudaFree(b->d_prm);
    b->d_states = nullptr;
    b->d_jobs = nullptr;
    b->d_chk = b->d_swp = nullptr;
    b->d_prm = nullptr;
}

// Job grid for a given walkers-per-CTA bound; larger lattices first.  Instances with at most
// `thread_sites` sites run one thread per walker: their CTAs take up to 32 x (warps per CTA)
// walkers, as many as shared memory holds (job.x carries the layout in bit 24).
static int build_jobs(rewl_batch_t b, int wpb, int thread_sites)
{
    const int n = (int)b->inst.size();
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return move_smem_per_walker(b->inst[x]->N, b->inst[x]->W) >
               move_smem_per_walker(b->inst[y]->N, b->inst[y]->W);
    });
    auto threaded = [&](const rewl_t r) { return r->N <= thread_sites; };
    // warps per CTA: the bound, lowered where a warp-per-walker lattice needs it
    int gmax = 1;
    bool any_warp = false;
    for (int i : order) {
        const rewl_t r = b->inst[i];
        if (threaded(r)) continue;
        any_warp = true;
        const size_t per = move_smem_per_walker(r->N, r->W);
        gmax = std::max(gmax, std::max(1, std::min(wpb, (int)(MAX_SMEM_PER_CTA / per))));
    }
    if (!any_warp) gmax = wpb;
    std::vector<int4> jobs;
    size_t smem = 0;
    for (int i : order) {
        const rewl_t r = b->inst[i];
        if (threaded(r)) {
            const size_t per = move_smem_per_thread_walker(r->N, r->W);
            const int g = std::max(1, std::min(32 * gmax, (int)(MAX_SMEM_PER_CTA / per)));
            for (int s0 = 0; s0 < r->nw; s0 += g) {
                const int cnt = std::min(g, r->nw - s0);
                jobs.push_back(make_int4(i | (1 << 24), s0, cnt, 0));
                smem = std::max(smem, (size_t)cnt * per);
            }
            continue;
        }
        const size_t per = move_smem_per_walker(r->N, r->W);
        const int g = std::max(1, std::min(wpb, (int)(MAX_SMEM_PER_CTA / per)));
        for (int s0 = 0; s0 < r->nw; s0 += g) {
            const int cnt = std::min(g, r->nw - s0);
            jobs.push_back(make_int4(i, s0, cnt, 0));
            smem = std::max(smem, (size_t)cnt * per);
        }
    }
    cudaFree(b->d_jobs);
    b->d_jobs = nullptr;
    cudaError_t e = cudaMalloc(&b->d_jobs, jobs.size() * sizeof(int4));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_jobs, jobs.data(), jobs.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return b->cuda_fail(e, "batch jobs");
    b->njobs = (int)jobs.size();
    b->block_walkers = gmax;
    b->smem = smem;
    b->wpb_used = wpb;
    b->thread_sites = thread_sites;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    return REWL_OK;
}

static int auto_wpb(rewl_batch_t b)
{
    long long nw = 0;
    for (rewl_t r : b->inst) nw += r->nw;
    int g = (int)((nw + b->sms - 1) / b->sms);
    int p = 1;
    while (p < g) p <<= 1;
    return std::min(p, 16);
}

static cudaError_t enqueue_batch_round(rewl_batch_t b)
{
    MoveCfg c{};
    c.T = (int)b->interval;
    c.walkers_per_block = b->block_walkers;
    c.check_all = b->check_all;
    c.eps_l = LNU32_EPS;
    cudaError_t e = cudaSuccess;
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (b->profile) {
        if (!b->ev_free.empty()) {
            ev = b->ev_free.back();
            b->ev_free.pop_back();
        } else {
            e = cudaEventCreate(&ev.first);
            if (e == cudaSuccess) e = cudaEventCreate(&ev.second);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev.first, b->stream);
    }
    if (e == cudaSuccess)
        e = launch_move_batch(b->d_states, b->d_jobs, b->njobs, b->block_walkers, b->smem, c, b->stream);
    if (b->profile && e == cudaSuccess) {
        e = cudaEventRecord(ev.second, b->stream);
        b->ev_used.push_back(ev);
    }
    const int n = (int)b->inst.size();
    if (e == cudaSuccess) e = launch_check_batch(b->d_states, b->d_chk, b->nchk, b->d_prm, b->stream);
    if (e == cudaSuccess) e = launch_swap_batch(b->d_states, b->d_swp, b->nswp, b->stream);
    if (e == cudaSuccess) e = launch_round_end_batch(b->d_states, n, b->stream);
    return e;
}

static int batch_status(rewl_batch_t b, int *all_done, int *any_err)
{
    const int n = (int)b->inst.size();
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(&b->h_status[i], b->inst[i]->st.status, sizeof(DevStatus),
                            cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b->cuda_fail(e, "batch status");
    int done = 1, err = 0;
    for (int i = 0; i < n; ++i) {
        done &= b->h_status[i].done;
        err |= b->h_status[i].err;
    }
    *all_done = done;
    *any_err = err;
    return REWL_OK;
}

extern "C" {

int rewl_batch_create(rewl_batch_t *out, const rewl_desc_t *d, int n, long long interval)
{
    if (!out || !d || n < 1 || n > 4096 || interval < 1 || interval > 100000000) {
        g_err = "rewl_batch_create: invalid argument";
        return REWL_ERR_INVALID_ARG;
    }
    *out = nullptr;
    rewl_batch_t b = new rewl_batch_s();
    b->interval = interval;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 0; i < n; ++i) {
        rewl_t r = nullptr;
        int rc = rewl_create(&r, d[i].model, d[i].L, d[i].windows, d[i].overlap,
                             d[i].walkers_per_window, d[i].lnf_final, d[i].flatness);
        if (rc == REWL_OK) rc = rewl_set_seed(r, d[i].seed);
        if (rc == REWL_OK) rc = rewl_set_param(r, "interval", (double)interval);
        if (rc == REWL_OK && d[i].lnf_init > 0.0) rc = rewl_set_param(r, "lnf_init", d[i].lnf_init);
        if (rc == REWL_OK) rc = rewl_set_param(r, "instance", (double)d[i].instance);
        if (rc != REWL_OK) {
            const std::string m = "rewl_batch_create: instance " + std::to_string(i) + ": " +
                                  rewl_last_error(r);
            if (r) rewl_destroy(r);
            for (rewl_t x : b->inst) rewl_destroy(x);
            delete b;
            g_err = m;
            return rc;
        }
        b->inst.push_back(r);
    }
    if (cudaHostAlloc((void **)&b->h_status, n * sizeof(DevStatus), cudaHostAllocDefault) != cudaSuccess) {
        for (rewl_t x : b->inst) rewl_destroy(x);
        delete b;
        g_err = "rewl_batch_create: pinned status allocation failed";
        return REWL_ERR_CUDA;
    }
    *out = b;
    return REWL_OK;
}

int rewl_batch_set_param(rewl_batch_t b, const char *key, double v)
{
    if (!b || !key) return REWL_ERR_INVALID_ARG;
    const std::string k(key);
    if (k == "walkers_per_block" && v >= 0 && v <= 16) {
        b->wpb = (int)v;
        return b->inited ? build_jobs(b, b->wpb > 0 ? b->wpb : auto_wpb(b), b->thread_sites) : REWL_OK;
    }
    if (k == "thread_layout_max_sites" && v >= 0 && v <= 65536) {
        b->thread_sites = (int)v;
        return b->inited ? build_jobs(b, b->wpb > 0 ? b->wpb : auto_wpb(b), b->thread_sites) : REWL_OK;
    }
    if (k == "graph_rounds" && v >= 0 && v <= 4096) {
        b->graph_rounds = (int)v;
        return REWL_OK;
    }
    if (k == "profile" && (v == 0 || v == 1)) {
        b->profile = (int)v;
        return REWL_OK;
    }
    if (k == "check_all" && (v == 0 || v == 1)) {
        b->check_all = (int)v;
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        return REWL_OK;
    }
    if (k == "prep_budget" && !b->inited) {
        for (rewl_t r : b->inst) {
            const int rc = rewl_set_param(r, key, v);
            if (rc != REWL_OK) return b->fail(rc, rewl_last_error(r));
        }
        return REWL_OK;
    }
    return b->fail(REWL_ERR_INVALID_ARG, "rewl_batch_set_param: unknown key or bad value: " + k);
}

int rewl_batch_set_stream(rewl_batch_t b, void *stream)
{
    if (!b) return REWL_ERR_INVALID_ARG;
    b->stream = (cudaStream_t)stream;
    for (rewl_t r : b->inst) rewl_set_stream(r, stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    return REWL_OK;
}

int rewl_batch_init(rewl_batch_t b)
{
    if (!b) return REWL_ERR_INVALID_ARG;
    const int n = (int)b->inst.size();
    for (int i = 0; i < n; ++i) {
        rewl_set_stream(b->inst[i], b->stream);
        const int rc = rewl_init(b->inst[i]);
        if (rc != REWL_OK)
            return b->fail(rc, "instance " + std::to_string(i) + ": " + rewl_last_error(b->inst[i]));
    }
    free_tables(b);
    std::vector<State> states(n);
    std::vector<int2> chk, swp;
    std::vector<double2> prm(n);
    for (int i = 0; i < n; ++i) {
        const rewl_t r = b->inst[i];
        states[i] = r->st;
        prm[i] = make_double2(r->flatness, r->lnf_final);
        for (int w = 0; w < r->h; ++w) chk.push_back(make_int2(i, w));
        for (int p = 0; p < (r->h + 1) / 2 && r->h > 1; ++p) swp.push_back(make_int2(i, p));
    }
    cudaError_t e = cudaMalloc(&b->d_states, n * sizeof(State));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_prm, n * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_chk, std::max<size_t>(1, chk.size()) * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_swp, std::max<size_t>(1, swp.size()) * sizeof(int2));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_states, states.data(), n * sizeof(State), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_prm, prm.data(), n * sizeof(double2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !chk.empty())
        e = cudaMemcpy(b->d_chk, chk.data(), chk.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !swp.empty())
        e = cudaMemcpy(b->d_swp, swp.data(), swp.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return b->cuda_fail(e, "rewl_batch_init tables");
    b->nchk = (int)chk.size();
    b->nswp = (int)swp.size();
    const int rc = build_jobs(b, b->wpb > 0 ? b->wpb : auto_wpb(b), b->thread_sites);
    if (rc != REWL_OK) return rc;
    b->inited = true;
    b->seconds = 0.0;
    return REWL_OK;
}

int rewl_batch_step(rewl_batch_t b, int rounds)
{
    if (!b || rounds < 0) return REWL_ERR_INVALID_ARG;
    if (!b->inited) return b->fail(REWL_ERR_STATE, "rewl_batch_step before rewl_batch_init");
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < rounds && e == cudaSuccess; ++i) e = enqueue_batch_round(b);
    if (e != cudaSuccess) return b->cuda_fail(e, "rewl_batch_step");
    return REWL_OK;
}

static int build_batch_graph(rewl_batch_t b, int len)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return b->cuda_fail(e, "graph stream");
    cudaStream_t saved = b->stream;
    const int prof = b->profile;
    b->stream = cap;
    b->profile = 0;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    for (int i = 0; i < len && e == cudaSuccess; ++i) e = enqueue_batch_round(b);
    const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    b->stream = saved;
    b->profile = prof;
    cudaStreamDestroy(cap);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return b->cuda_fail(e, "batch graph capture");
    }
    b->graph_len = len;
    return REWL_OK;
}

int rewl_batch_run(rewl_batch_t b, double max_seconds, long long max_rounds, int *status)
{
    if (!b) return REWL_ERR_INVALID_ARG;
    if (status) *status = REWL_STATUS_RUNNING;
    if (!b->inited) {
        const int rc = rewl_batch_init(b);
        if (rc != REWL_OK) return rc;
    }
    const auto t0 = std::chrono::steady_clock::now();
    long long launched = 0;
    int chunk = 1, rc = REWL_OK, st_out = REWL_STATUS_RUNNING;
    for (;;) {
        int done = 0, err = 0;
        rc = batch_status(b, &done, &err);
        if (rc != REWL_OK) break;
        if (err) {
            rc = b->fail(REWL_ERR_STATE, "device error flags " + std::to_string(err));
            break;
        }
        if (done) {
            st_out = REWL_STATUS_DONE;
            break;
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if ((max_rounds >= 0 && launched >= max_rounds) || (max_seconds > 0 && el >= max_seconds)) {
            st_out = REWL_STATUS_BUDGET;
            break;
        }
        long long n = chunk;
        if (max_rounds >= 0) n = std::min(n, max_rounds - launched);
        cudaError_t e = cudaSuccess;
        const int gl = b->graph_rounds;
        if (gl > 0 && n >= gl && !b->profile) {
            if (!b->graph || b->graph_len != gl) {
                rc = build_batch_graph(b, gl);
                if (rc != REWL_OK) break;
            }
            n = gl;
            e = cudaGraphLaunch(b->graph, b->stream);
        } else {
            for (long long i = 0; i < n && e == cudaSuccess; ++i) e = enqueue_batch_round(b);
        }
        if (e != cudaSuccess) {
            rc = b->cuda_fail(e, "rewl_batch_run launch");
            break;
        }
        launched += n;
        const auto tc = std::chrono::steady_clock::now();
        cudaError_t es = cudaStreamSynchronize(b->stream);
        if (es != cudaSuccess) {
            rc = b->cuda_fail(es, "rewl_batch_run");
            break;
        }
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - tc).count();
        if (dt < 0.05 && chunk < 4096) chunk *= 2;
    }
    b->seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (status) *status = st_out;
    return rc;
}

int rewl_batch_autotune(rewl_batch_t b, int rounds, int *best, double *ms)
{
    if (!b || rounds < 1) return REWL_ERR_INVALID_ARG;
    if (!b->inited) {
        const int rc = rewl_batch_init(b);
        if (rc != REWL_OK) return rc;
    }
    // the trial rounds are rounds of the simulation itself: results do not depend on the
    // launch configuration, so timing candidates costs nothing but the choice.
    // 1) layout x walkers per CTA: per-round time of `rounds` rounds for every pair
    static const int wcand[4] = {2, 4, 8, 16};
    static const int tcand[4] = {0, 400, 1024, 1600};
    static const int gcand[3] = {8, 32, 128};
    double bestms = 1e300;
    int bestg = 4, bestt = 0, bestgr = b->graph_rounds;
    cudaEvent_t a = nullptr, z = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&z);
    if (e != cudaSuccess) return b->cuda_fail(e, "autotune events");
    int rc = REWL_OK;
    const int prof = b->profile;
    b->profile = 0;
    auto timed = [&](int nrounds, bool graph, double *per) -> int {
        cudaError_t e2 = cudaEventRecord(a, b->stream);
        if (graph) {
            for (int i = 0; i < nrounds / b->graph_len && e2 == cudaSuccess; ++i)
                e2 = cudaGraphLaunch(b->graph, b->stream);
        } else {
            for (int i = 0; i < nrounds && e2 == cudaSuccess; ++i) e2 = enqueue_batch_round(b);
        }
        if (e2 == cudaSuccess) e2 = cudaEventRecord(z, b->stream);
        if (e2 == cudaSuccess) e2 = cudaEventSynchronize(z);
        float t = 0.f;
        if (e2 == cudaSuccess) e2 = cudaEventElapsedTime(&t, a, z);
        if (e2 != cudaSuccess) return b->cuda_fail(e2, "autotune");
        *per = (double)t / nrounds;
        return REWL_OK;
    };
    int ci = 0;
    for (int ti = 0; ti < 4 && rc == REWL_OK; ++ti)
        for (int wi = 0; wi < 4 && rc == REWL_OK; ++wi, ++ci) {
            bool any_thread = false;
            for (rewl_t r : b->inst) any_thread |= r->N <= tcand[ti];
            double per = 1e300;
            if (ti == 0 || any_thread) { // a threshold no instance reaches repeats candidate ti = 0
                rc = build_jobs(b, wcand[wi], tcand[ti]);
                if (rc == REWL_OK) rc = timed(rounds, false, &per);
            }
            if (ms) ms[ci] = per < 1e300 ? per : -1.0;
            if (rc == REWL_OK && per < bestms) {
                bestms = per;
                bestg = wcand[wi];
                bestt = tcand[ti];
            }
        }
    // 2) rounds per CUDA-graph replay, with the chosen layout
    if (rc == REWL_OK) rc = build_jobs(b, bestg, bestt);
    double bestgms = 1e300;
    for (int gi = 0; gi < 3 && rc == REWL_OK; ++gi, ++ci) {
        rc = build_batch_graph(b, gcand[gi]);
        double per = 1e300;
        if (rc == REWL_OK) rc = timed(gcand[gi], true, &per);
        if (ms) ms[ci] = rc == REWL_OK ? per : -1.0;
        if (rc == REWL_OK && per < bestgms) {
            bestgms = per;
            bestgr = gcand[gi];
        }
    }
    b->profile = prof;
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    if (rc != REWL_OK) return rc;
    b->wpb = bestg;
    b->graph_rounds = bestgr;
    if (best) {
        best[0] = bestg;
        best[1] = bestt;
        best[2] = bestgr;
    }
    return build_jobs(b, bestg, bestt);
}

int rewl_batch_instance(rewl_batch_t b, int i, rewl_t *out)
{
    if (!b || !out || i < 0 || i >= (int)b->inst.size()) return REWL_ERR_INVALID_ARG;
    *out = b->inst[i];
    return REWL_OK;
}

int rewl_batch_info(rewl_batch_t b, int *out)
{
    if (!b || !out) return REWL_ERR_INVALID_ARG;
    long long nw = 0;
    for (rewl_t r : b->inst) nw += r->nw;
    out[0] = (int)b->inst.size();
    out[1] = (int)nw;
    out[2] = b->njobs;
    out[3] = b->block_walkers;
    out[4] = b->thread_sites;
    out[5] = b->graph_rounds;
    return REWL_OK;
}

int rewl_batch_kernel_time(rewl_batch_t b, double *move_ms, long long *launches, int reset)
{
    if (!b) return REWL_ERR_INVALID_ARG;
    double tot = 0.0;
    for (auto &ev : b->ev_used) {
        cudaError_t e = cudaEventSynchronize(ev.second);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.first, ev.second);
        if (e != cudaSuccess) return b->cuda_fail(e, "rewl_batch_kernel_time");
        tot += ms;
    }
    if (move_ms) *move_ms = tot;
    if (launches) *launches = (long long)b->ev_used.size();
    if (reset) {
        for (auto &ev : b->ev_used) b->ev_free.push_back(ev);
        b->ev_used.clear();
    }
    return REWL_OK;
}

void rewl_batch_destroy(rewl_batch_t b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto *v : {&b->ev_used, &b->ev_free})
        for (auto &ev : *v) {
            cudaEventDestroy(ev.first);
            cudaEventDestroy(ev.second);
        }
    free_tables(b);
    if (b->h_status) cudaFreeHost(b->h_status);
    for (rewl_t r : b->inst) rewl_destroy(r);
    delete b;
}

const char *rewl_batch_last_error(rewl_batch_t b)
{
    if (b) return b->err.c_str();
    return g_err.c_str();
}

} // extern "C"
