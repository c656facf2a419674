// rewl_host.cu -- host runtime behind include/rewl.h: handle lifecycle, device state, the
// round loop (move kernel, flatness/advance, exchange, round end) captured in CUDA graphs,
// joining, state access, statistics and checkpoints.  No method arithmetic runs on the host.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "rewl.h"
#include "rewl_device.cuh"
#include "rewl_kernels.cuh"
#include "rewl_handle.h"

using namespace rewl;

thread_local std::string g_err; // message of the last failed call without a handle

namespace {

template <typename T> T *dmalloc(size_t n, cudaError_t &e)
{
    void *p = nullptr;
    if (e != cudaSuccess) return nullptr;
    e = cudaMalloc(&p, (n ? n : 1) * sizeof(T));
    if (e == cudaSuccess) e = cudaMemset(p, 0, (n ? n : 1) * sizeof(T));
    return static_cast<T *>(p);
}

// Equal-size windows with overlap o (Fig. 1a); see rewl_create in rewl.h.
int make_windows(int B, int h, double o, std::vector<int> &lo, std::vector<int> &hi)
{
    if (B < 1 || h < 1 || !(o >= 0.0 && o < 1.0)) return -1;
    lo.assign(h, 0);
    hi.assign(h, B);
    if (h == 1) return 0;
    if (o == 0.75) {
        const long long den = 2LL * (h + 3);
        for (int k = 0; k < h; ++k) {
            lo[k] = (int)((2LL * k * B + (h + 3)) / den);
            hi[k] = (int)std::min<long long>(B, (2LL * (k + 4) * B + (h + 3)) / den);
        }
    } else {
        const double W = (double)B / (1.0 + (double)(h - 1) * (1.0 - o));
        const double s = (1.0 - o) * W;
        for (int k = 0; k < h; ++k) {
            lo[k] = (int)std::floor((double)k * s + 0.5);
            hi[k] = (int)std::min((double)B, std::floor((double)k * s + W + 0.5));
        }
    }
    hi[h - 1] = B;
    for (int k = 0; k + 1 < h; ++k)
        if (lo[k + 1] > hi[k] || lo[k + 1] <= lo[k]) return -2;
    return 0;
}

int check_windows(int B, const std::vector<int> &lo, const std::vector<int> &hi)
{
    const int h = (int)lo.size();
    if (h < 1 || lo[0] != 0 || hi[h - 1] != B) return -1;
    for (int k = 0; k < h; ++k)
        if (lo[k] > hi[k]) return -1;
    for (int k = 0; k + 1 < h; ++k)
        if (lo[k + 1] > hi[k] || lo[k + 1] <= lo[k] || hi[k + 1] <= hi[k]) return -1;
    return 0;
}

} // namespace

static int walkers_per_block(const rewl_t r)
{
    const size_t per = move_smem_per_walker(r->N, r->W);
    int g = r->wpb;
    if (g <= 0) { // one warp per SM sub-partition first; beyond 4 walkers per SM, more CTAs of
                  // 4 (measured: 8 or 16 per CTA is slower than 4 for 1024 walkers)
        g = (r->nw + r->sms - 1) / r->sms;
        int p = 1;
        while (p < g) p <<= 1;
        g = std::min(p, 4);
    }
    while (g > 1 && (size_t)g * per > MAX_SMEM_PER_CTA) g >>= 1;
    return g;
}

// walkers (threads) per CTA of the thread-per-walker layout: whole warps, spread over the SMs,
// at most 128 and what shared memory holds
static int thread_walkers_per_block(const rewl_t r)
{
    const size_t per = move_smem_per_thread_walker(r->N, r->W);
    int g = (r->nw + r->sms - 1) / r->sms;
    g = std::min(128, std::max(32, (g + 31) & ~31));
    while (g > 1 && (size_t)g * per > MAX_SMEM_PER_CTA) --g;
    return g;
}

static void release(rewl_t r)
{
    if (r->graph) cudaGraphExecDestroy(r->graph);
    r->graph = nullptr;
    State &s = r->st;
    void *ptrs[] = {s.spins, s.cfg, s.k, s.lng, s.H, s.step, s.acc, s.pstep, s.restarts, s.flat,
                    r->d_lohi, s.lnf, s.iter, s.finished, s.mask, s.swap_att, s.swap_acc,
                    s.it1_round, s.mode, s.frag, s.hem, s.status, r->d_mean, r->d_out, r->d_joins,
                    r->d_ok};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (r->h_status) cudaFreeHost(r->h_status);
    r->h_status = nullptr;
    r->st = State{};
    r->d_lohi = nullptr;
    r->d_mean = r->d_out = nullptr;
    r->d_joins = r->d_ok = nullptr;
    r->allocated = false;
}

static int allocate(rewl_t r)
{
    if (r->allocated) release(r);
    r->h = (int)r->lo.size();
    r->nw = r->h * r->m;
    r->W = 0;
    for (int w = 0; w < r->h; ++w) r->W = std::max(r->W, r->hi[w] - r->lo[w] + 1);
    State &s = r->st;
    cudaError_t e = cudaSuccess;
    const size_t nw = (size_t)r->nw, W = (size_t)r->W, h = (size_t)r->h;
    s.model = r->model;
    s.production = r->production;
    s.w0 = r->w_begin;
    s.slot0 = r->w_begin * r->m;
    s.q = r->q;
    s.L = r->L;
    s.N = r->N;
    s.nw = r->nw;
    s.m = r->m;
    s.h = r->h;
    s.W = r->W;
    s.spin_stride = (r->N + 15) & ~15;
    s.vec_spins = (r->N & 15) == 0;
    s.magic = (uint32_t)((0x100000000ULL + (uint64_t)r->L - 1) / (uint64_t)r->L);
    if (move_smem_per_walker(r->N, r->W) > MAX_SMEM_PER_CTA)
        return r->fail(REWL_ERR_INVALID_ARG, "lattice and window do not fit in shared memory");
    s.spins = dmalloc<int8_t>(nw * s.spin_stride, e);
    s.cfg = dmalloc<int>(nw, e);
    s.k = dmalloc<int>(nw, e);
    s.lng = dmalloc<double>(nw * W, e);
    s.H = dmalloc<uint32_t>(nw * W, e);
    s.step = dmalloc<unsigned long long>(nw, e);
    s.acc = dmalloc<unsigned long long>(nw, e);
    s.pstep = dmalloc<unsigned long long>(nw, e);
    s.restarts = dmalloc<int>(nw, e);
    s.flat = dmalloc<uint8_t>(nw, e);
    r->d_lohi = dmalloc<int>(2 * h, e);
    s.lnf = dmalloc<double>(h, e);
    s.iter = dmalloc<int>(h, e);
    s.finished = dmalloc<uint8_t>(h, e);
    s.mask = dmalloc<uint8_t>(h * W, e);
    s.swap_att = dmalloc<unsigned long long>(h, e);
    s.swap_acc = dmalloc<unsigned long long>(h, e);
    s.it1_round = dmalloc<long long>(h, e);
    s.mode = dmalloc<uint8_t>(h, e);
    s.frag = dmalloc<double>(nw * W, e);
    s.status = dmalloc<DevStatus>(1, e);
    r->d_mean = dmalloc<double>(h * W, e);
    r->d_out = dmalloc<double>((size_t)r->B + 1, e);
    r->d_joins = dmalloc<int>(h, e);
    r->d_ok = dmalloc<int>(1, e);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&r->h_status, sizeof(DevStatus), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        release(r);
        return r->cuda_fail(e, "allocate");
    }
    s.lo = r->d_lohi;
    s.hi = r->d_lohi + h;
    s.key0 = (uint32_t)r->seed;
    s.key1 = (uint32_t)(r->seed >> 32);
    s.inst = r->inst;
    r->allocated = true;
    // host-side validation of the site -> (x, y) multiply-high
    for (uint32_t site = 0; site < (uint32_t)r->N; ++site)
        if ((uint32_t)(((uint64_t)site * s.magic) >> 32) != site / (uint32_t)r->L)
            return r->fail(REWL_ERR_INVALID_ARG, "lattice too large for the site decomposition");
    return REWL_OK;
}

extern "C" {

int rewl_create(rewl_t *out, int model, int L, int windows, double overlap, int walkers_per_window,
                double lnf_final, double flatness)
{
    if (!out) {
        g_err = "rewl_create: out is NULL";
        return REWL_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (L < 2 || L > 255 || (model != 0 && (model < 2 || model > 127)) || windows < 1 ||
        walkers_per_window < 1 || walkers_per_window > MAX_M || !(lnf_final >= 0x1p-32) ||
        !(flatness >= 0.0) || (long long)windows * walkers_per_window > (1LL << 24)) {
        g_err = "rewl_create: invalid argument";
        return REWL_ERR_INVALID_ARG;
    }
    rewl_t r = new rewl_s();
    r->model = model;
    r->q = model == 0 ? 2 : model;
    r->L = L;
    r->N = L * L;
    r->B = model == 0 ? r->N : 2 * r->N;
    r->m = walkers_per_window;
    r->overlap = overlap;
    r->lnf_final = lnf_final;
    r->flatness = flatness;
    if (make_windows(r->B, windows, overlap, r->lo, r->hi) != 0) {
        delete r;
        g_err = "rewl_create: windows do not overlap (too many windows or bad overlap)";
        return REWL_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&r->sms, cudaDevAttrMultiProcessorCount, dev);
    const int rc = allocate(r);
    if (rc != REWL_OK) {
        g_err = r->err;
        delete r;
        return rc;
    }
    *out = r;
    return REWL_OK;
}

int rewl_set_param(rewl_t r, const char *key, double v)
{
    if (!r || !key) return REWL_ERR_INVALID_ARG;
    const std::string k(key);
    if (k == "profile" && (v == 0 || v == 1)) {
        r->profile = (int)v;
        return REWL_OK;
    }
    if (k == "production" && (v == 0 || v == 1)) {
        if (r->shard && v == 0)
            return r->fail(REWL_ERR_INVALID_ARG, "production: a shard never ends a run by itself");
        r->production = (int)v;
        r->st.production = (int)v;
        if (r->graph) cudaGraphExecDestroy(r->graph);
        r->graph = nullptr;
        if (r->inited) { // re-evaluate "every window finished" under the new rule
            cudaError_t e = launch_set_done(r->st, r->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
            if (e != cudaSuccess) return r->cuda_fail(e, "rewl_set_param(production)");
        }
        return REWL_OK;
    }
    if (k == "measure_em" && (v == 0 || v == 1)) {
        if (r->model != 0) return r->fail(REWL_ERR_INVALID_ARG, "measure_em: Ising model only");
        if (!r->allocated) return r->fail(REWL_ERR_STATE, "measure_em: no state");
        const size_t N1 = (size_t)r->N + 1;
        if ((size_t)r->h * r->W * N1 > (1u << 30) || (size_t)(r->B + 1) * N1 > (1u << 28))
            return r->fail(REWL_ERR_INVALID_ARG, "measure_em: lattice too large for the (E, M) grid");
        if (r->graph) cudaGraphExecDestroy(r->graph);
        r->graph = nullptr;
        cudaError_t e = cudaStreamSynchronize(r->stream);
        if (r->st.hem) cudaFree(r->st.hem);
        r->st.hem = nullptr;
        if (v == 1 && e == cudaSuccess) {
            const size_t bytes = (size_t)r->h * r->W * N1 * 4u;
            e = cudaMalloc(&r->st.hem, bytes);
            if (e == cudaSuccess) e = cudaMemsetAsync(r->st.hem, 0, bytes, r->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
        }
        if (e != cudaSuccess) return r->cuda_fail(e, "rewl_set_param(measure_em)");
        return REWL_OK;
    }
    if (r->inited) return r->fail(REWL_ERR_STATE, "rewl_set_param after rewl_init");
    // the move kernel's int64 ln g shadow needs 2^-32 <= ln f < 2^20 and interval * ln f < 2^30
    if (k == "lnf_init" && v >= 0x1p-32 && v < 0x1p20 && v * (double)r->interval < 0x1p30) r->lnf_init = v;
    else if (k == "interval" && v >= 1 && v <= 1e8 && std::floor(v) * r->lnf_init < 0x1p30)
        r->interval = (long long)v;
    else if (k == "prep_budget" && v >= 1 && v <= 1e9) r->prep_budget = (long long)v;
    else if (k == "instance" && v >= 0 && v < 16777216.0) r->inst = (uint32_t)v;
    else if (k == "graph_rounds" && v >= 0 && v <= 4096) r->graph_rounds = (int)v;
    else if (k == "walkers_per_block" && v >= 0 && v <= 16) r->wpb = (int)v;
    else if (k == "check_all" && (v == 0 || v == 1)) r->check_all = (int)v;
    else if (k == "layout" && (v == 0 || v == 1)) r->layout = (int)v;
    else if (k == "schedule" && (v == 0 || v == 1)) r->schedule = (int)v;
    else return r->fail(REWL_ERR_INVALID_ARG, "rewl_set_param: unknown key or bad value: " + k);
    if (k == "instance") r->st.inst = r->inst;
    return REWL_OK;
}

int rewl_set_seed(rewl_t r, uint64_t seed)
{
    if (!r) return REWL_ERR_INVALID_ARG;
    if (r->inited) return r->fail(REWL_ERR_STATE, "rewl_set_seed after rewl_init");
    r->seed = seed;
    r->st.key0 = (uint32_t)seed;
    r->st.key1 = (uint32_t)(seed >> 32);
    return REWL_OK;
}

int rewl_set_lng_init(rewl_t r, const double *lng, int n)
{
    if (!r || !lng) return REWL_ERR_INVALID_ARG;
    if (r->inited) return r->fail(REWL_ERR_STATE, "rewl_set_lng_init after rewl_init");
    if (n != r->B + 1) return r->fail(REWL_ERR_INVALID_ARG, "rewl_set_lng_init: n must be B+1");
    for (int b = 0; b <= r->B; ++b)
        if (!std::isfinite(lng[b]))
            return r->fail(REWL_ERR_INVALID_ARG, "rewl_set_lng_init: non-finite ln g");
    r->lng_init.assign(lng, lng + n);
    return REWL_OK;
}

int rewl_set_windows(rewl_t r, const int *lo_hi, int h)
{
    if (!r || !lo_hi || h < 1) return REWL_ERR_INVALID_ARG;
    if (r->inited) return r->fail(REWL_ERR_STATE, "rewl_set_windows after rewl_init");
    if (r->shard) return r->fail(REWL_ERR_STATE, "rewl_set_windows on a shard (use rewl_set_shard)");
    std::vector<int> lo(lo_hi, lo_hi + h), hi(lo_hi + h, lo_hi + 2 * h);
    if (check_windows(r->B, lo, hi) != 0)
        return r->fail(REWL_ERR_INVALID_ARG, "rewl_set_windows: invalid layout");
    if ((long long)h * r->m > (1LL << 24)) return r->fail(REWL_ERR_INVALID_ARG, "too many walkers");
    r->lo = lo;
    r->hi = hi;
    return allocate(r);
}

int rewl_set_shard(rewl_t r, const int *lo_hi, int h_global, int w_begin)
{
    if (!r || !lo_hi || h_global < 2) return REWL_ERR_INVALID_ARG;
    if (r->inited) return r->fail(REWL_ERR_STATE, "rewl_set_shard after rewl_init");
    const int hl = r->shard ? (int)r->lo.size() : r->h;
    std::vector<int> lo(lo_hi, lo_hi + h_global), hi(lo_hi + h_global, lo_hi + 2 * h_global);
    if (check_windows(r->B, lo, hi) != 0)
        return r->fail(REWL_ERR_INVALID_ARG, "rewl_set_shard: invalid global layout");
    if (w_begin < 0 || w_begin + hl > h_global || hl >= h_global)
        return r->fail(REWL_ERR_INVALID_ARG, "rewl_set_shard: windows outside the global layout");
    if ((long long)h_global * r->m > (1LL << 24)) return r->fail(REWL_ERR_INVALID_ARG, "too many walkers");
    r->lo.assign(lo.begin() + w_begin, lo.begin() + w_begin + hl);
    r->hi.assign(hi.begin() + w_begin, hi.begin() + w_begin + hl);
    const int we = w_begin + hl;
    r->nbr[0] = w_begin > 0 ? lo[w_begin - 1] : -1;
    r->nbr[1] = w_begin > 0 ? hi[w_begin - 1] : -1;
    r->nbr[2] = we < h_global ? lo[we] : -1;
    r->nbr[3] = we < h_global ? hi[we] : -1;
    r->shard = 1;
    r->w_begin = w_begin;
    r->production = 1; // only the caller sees every shard: it decides when the run ends
    return allocate(r);
}

static int bnd_check(rewl_t r, int side)
{
    if (!r->shard) return r->fail(REWL_ERR_STATE, "boundary exchange: not a shard (rewl_set_shard)");
    if (!r->inited) return r->fail(REWL_ERR_STATE, "boundary exchange before rewl_init");
    if (side != 0 && side != 1) return r->fail(REWL_ERR_INVALID_ARG, "boundary exchange: side must be 0 or 1");
    if (r->nbr[2 * side] < 0)
        return r->fail(REWL_ERR_INVALID_ARG, "boundary exchange: no neighbouring shard on that side");
    return REWL_OK;
}

int rewl_boundary_bins(rewl_t r, int side, int *bins)
{
    if (!r || !bins) return REWL_ERR_INVALID_ARG;
    int rc = bnd_check(r, side);
    if (rc != REWL_OK) return rc;
    cudaError_t e = launch_bnd_bins(r->st, side, bins, r->stream);
    return e == cudaSuccess ? REWL_OK : r->cuda_fail(e, "rewl_boundary_bins");
}

int rewl_boundary_half(rewl_t r, int side, const int *partner_bins, double *half)
{
    if (!r || !partner_bins || !half) return REWL_ERR_INVALID_ARG;
    int rc = bnd_check(r, side);
    if (rc != REWL_OK) return rc;
    const int plo = side ? r->nbr[2] : r->nbr[0], phi = side ? r->nbr[3] : r->nbr[1];
    cudaError_t e = launch_bnd_half(r->st, side, plo, phi, partner_bins, half, r->stream);
    return e == cudaSuccess ? REWL_OK : r->cuda_fail(e, "rewl_boundary_half");
}

int rewl_boundary_decide(rewl_t r, int side, const double *half, const double *partner_half,
                         uint8_t *accepted, int8_t *lattices)
{
    if (!r || !half || !partner_half || !accepted || !lattices) return REWL_ERR_INVALID_ARG;
    int rc = bnd_check(r, side);
    if (rc != REWL_OK) return rc;
    cudaError_t e = launch_bnd_decide(r->st, side, half, partner_half, accepted, lattices, r->stream);
    return e == cudaSuccess ? REWL_OK : r->cuda_fail(e, "rewl_boundary_decide");
}

int rewl_boundary_import(rewl_t r, int side, const int *partner_bins, const uint8_t *accepted,
                         const int8_t *partner_lattices)
{
    if (!r || !partner_bins || !accepted || !partner_lattices) return REWL_ERR_INVALID_ARG;
    int rc = bnd_check(r, side);
    if (rc != REWL_OK) return rc;
    cudaError_t e = launch_bnd_import(r->st, side, partner_bins, accepted, partner_lattices, r->stream);
    return e == cudaSuccess ? REWL_OK : r->cuda_fail(e, "rewl_boundary_import");
}

int rewl_set_stream(rewl_t r, void *stream)
{
    if (!r) return REWL_ERR_INVALID_ARG;
    if (r->graph) cudaGraphExecDestroy(r->graph);
    r->graph = nullptr;
    r->stream = (cudaStream_t)stream;
    return REWL_OK;
}

static int sync_status(rewl_t r)
{
    cudaError_t e = cudaMemcpyAsync(r->h_status, r->st.status, sizeof(DevStatus),
                                    cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return r->cuda_fail(e, "status");
    return REWL_OK;
}

int rewl_init(rewl_t r)
{
    if (!r) return REWL_ERR_INVALID_ARG;
    State &s = r->st;
    cudaStream_t st = r->stream;
    cudaError_t e = cudaSuccess;
    const size_t h = (size_t)r->h, W = (size_t)r->W;
    std::vector<int> lohi(2 * h);
    for (size_t w = 0; w < h; ++w) {
        lohi[w] = r->lo[w];
        lohi[h + w] = r->hi[w];
    }
    // per-walker initial ln g (0, or the warm start)
    std::vector<double> lng(h * r->m * W, 0.0);
    if (!r->lng_init.empty())
        for (size_t w = 0; w < h; ++w)
            for (int i = 0; i < r->m; ++i)
                for (int b = r->lo[w]; b <= r->hi[w]; ++b)
                    lng[(w * r->m + i) * W + (b - r->lo[w])] = r->lng_init[b];
    std::vector<double> lnf(h, r->lnf_init);
    std::vector<uint8_t> fin(h, (uint8_t)(r->lnf_init < r->lnf_final));
    e = cudaMemcpyAsync(r->d_lohi, lohi.data(), lohi.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.lng, lng.data(), lng.size() * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.lnf, lnf.data(), h * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.finished, fin.data(), h, cudaMemcpyHostToDevice, st);
    const size_t nw = (size_t)r->nw;
    if (e == cudaSuccess) e = cudaMemsetAsync(s.H, 0, nw * W * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.step, 0, nw * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.acc, 0, nw * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.flat, 0, nw, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.iter, 0, h * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.mask, 0, h * W, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.swap_att, 0, h * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.swap_acc, 0, h * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.it1_round, 0, h * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.mode, 0, h, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.frag, 0, nw * W * 8, st);
    s.schedule = r->schedule;
    if (e == cudaSuccess) e = cudaMemsetAsync(s.status, 0, sizeof(DevStatus), st);
    if (e == cudaSuccess) e = launch_init_prep(s, r->prep_budget, st);
    if (e == cudaSuccess) e = launch_set_done(s, st);
    if (e != cudaSuccess) return r->cuda_fail(e, "rewl_init");
    int rc = sync_status(r);
    if (rc != REWL_OK) return rc;
    r->inited = true;
    r->seconds = 0.0;
    if (r->h_status->err & ERR_PREP)
        return r->fail(REWL_ERR_PREP, "rewl_init: a walker could not reach its window");
    return REWL_OK;
}

cudaError_t rewl_enqueue_round(rewl_t r)
{
    MoveCfg c{};
    c.T = (int)r->interval;
    c.layout = r->layout;
    c.walkers_per_block = r->layout ? thread_walkers_per_block(r) : walkers_per_block(r);
    c.check_all = r->check_all;
    c.eps_l = LNU32_EPS;
    cudaError_t e = cudaSuccess;
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (r->profile) {
        if (!r->ev_free.empty()) {
            ev = r->ev_free.back();
            r->ev_free.pop_back();
        } else {
            e = cudaEventCreate(&ev.first);
            if (e == cudaSuccess) e = cudaEventCreate(&ev.second);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev.first, r->stream);
    }
    if (e == cudaSuccess) e = launch_move(r->st, c, r->stream);
    if (r->profile && e == cudaSuccess) {
        e = cudaEventRecord(ev.second, r->stream);
        r->ev_used.push_back(ev);
    }
    if (e == cudaSuccess && r->st.hem) e = launch_measure_em(r->st, r->stream);
    if (e == cudaSuccess) e = launch_check(r->st, r->flatness, r->lnf_final, r->stream);
    if (e == cudaSuccess) e = launch_swap(r->st, r->stream);
    if (e == cudaSuccess) e = launch_round_end(r->st, r->stream);
    return e;
}

static int build_graph(rewl_t r, int len)
{
    if (r->graph) cudaGraphExecDestroy(r->graph);
    r->graph = nullptr;
    cudaGraph_t g = nullptr;
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return r->cuda_fail(e, "graph stream");
    cudaStream_t saved = r->stream;
    r->stream = cap;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    const int prof = r->profile;
    r->profile = 0;
    for (int i = 0; i < len && e == cudaSuccess; ++i) e = rewl_enqueue_round(r);
    r->profile = prof;
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    r->stream = saved;
    cudaStreamDestroy(cap);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&r->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        r->graph = nullptr;
        return r->cuda_fail(e, "graph capture");
    }
    r->graph_len = len;
    return REWL_OK;
}

int rewl_run(rewl_t r, double max_seconds, long long max_rounds, int *status)
{
    if (!r) return REWL_ERR_INVALID_ARG;
    if (status) *status = REWL_STATUS_RUNNING;
    if (!r->inited) {
        const int rc = rewl_init(r);
        if (rc != REWL_OK) return rc;
    }
    r->abort_flag.store(0);
    const auto t0 = std::chrono::steady_clock::now();
    int rc = sync_status(r);
    if (rc != REWL_OK) return rc;
    const long long round0 = r->h_status->round;
    long long launched = 0;
    int chunk = 1;
    int st_out = REWL_STATUS_RUNNING;
    for (;;) {
        if (r->h_status->err) {
            rc = r->fail(REWL_ERR_STATE, "device error flags " + std::to_string(r->h_status->err));
            break;
        }
        if (r->h_status->done) {
            st_out = REWL_STATUS_DONE;
            break;
        }
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (max_rounds >= 0 && launched >= max_rounds) {
            st_out = REWL_STATUS_BUDGET;
            break;
        }
        if (max_seconds > 0 && el >= max_seconds) {
            st_out = REWL_STATUS_BUDGET;
            break;
        }
        if (r->abort_flag.load()) {
            st_out = REWL_STATUS_ABORTED;
            break;
        }
        long long n = chunk;
        if (max_rounds >= 0) n = std::min(n, max_rounds - launched);
        cudaError_t e = cudaSuccess;
        const int gl = r->graph_rounds;
        if (gl > 0 && n >= gl && !r->profile) {
            if (!r->graph || r->graph_len != gl) {
                rc = build_graph(r, gl);
                if (rc != REWL_OK) break;
            }
            n = gl;
            e = cudaGraphLaunch(r->graph, r->stream);
        } else {
            for (long long i = 0; i < n && e == cudaSuccess; ++i) e = rewl_enqueue_round(r);
        }
        if (e != cudaSuccess) {
            rc = r->cuda_fail(e, "rewl_run launch");
            break;
        }
        launched += n;
        const auto tc = std::chrono::steady_clock::now();
        rc = sync_status(r);
        if (rc != REWL_OK) break;
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - tc).count();
        if (dt < 0.05 && chunk < 4096) chunk *= 2; // grow the chunk while it stays short
    }
    r->seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    (void)round0;
    if (status) *status = st_out;
    return rc;
}

int rewl_step(rewl_t r, int rounds)
{
    if (!r || rounds < 0) return REWL_ERR_INVALID_ARG;
    if (!r->inited) return r->fail(REWL_ERR_STATE, "rewl_step before rewl_init");
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < rounds && e == cudaSuccess; ++i) e = rewl_enqueue_round(r);
    if (e != cudaSuccess) return r->cuda_fail(e, "rewl_step");
    return REWL_OK;
}

int rewl_kernel_time(rewl_t r, double *move_ms, long long *launches, int reset)
{
    if (!r) return REWL_ERR_INVALID_ARG;
    double tot = 0.0;
    for (auto &ev : r->ev_used) {
        cudaError_t e = cudaEventSynchronize(ev.second);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.first, ev.second);
        if (e != cudaSuccess) return r->cuda_fail(e, "rewl_kernel_time");
        tot += ms;
    }
    if (move_ms) *move_ms = tot;
    if (launches) *launches = (long long)r->ev_used.size();
    if (reset) {
        for (auto &ev : r->ev_used) r->ev_free.push_back(ev);
        r->ev_used.clear();
    }
    return REWL_OK;
}

int rewl_abort(rewl_t r)
{
    if (!r) return REWL_ERR_INVALID_ARG;
    r->abort_flag.store(1);
    return REWL_OK;
}

int rewl_jackknife(rewl_t r, double *err, int cap, int norm)
{
    if (!r || !err || (norm != 0 && norm != 1)) return REWL_ERR_INVALID_ARG;
    if (cap < r->B + 1) return r->fail(REWL_ERR_BUFFER_TOO_SMALL, "rewl_jackknife: cap < B+1");
    if (r->m < 2) return r->fail(REWL_ERR_STATE, "rewl_jackknife: needs at least 2 walkers per window");
    std::vector<uint8_t> fin((size_t)r->h);
    int rc = rewl_get_state(r, "finished", fin.data(), fin.size());
    if (rc != REWL_OK) return rc;
    for (uint8_t f : fin)
        if (!f) return r->fail(REWL_ERR_STATE, "rewl_jackknife: every window must be finished");
    const double de = r->model == 0 ? 4.0 : 1.0;
    const int step = (r->model != 0 && r->q == 2) ? 2 : 1;
    const double target = norm == 0 ? (double)r->N * std::log((double)r->q) : std::log((double)r->q);
    double *theta = nullptr, *d_err = nullptr;
    cudaError_t e = cudaMalloc(&theta, (size_t)r->m * (r->B + 1) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_err, (size_t)(r->B + 1) * 8);
    std::vector<int> oks((size_t)r->m, 0);
    for (int j = 0; j < r->m && e == cudaSuccess; ++j) {
        e = launch_loo_mean(r->st, j, r->d_mean, r->stream);
        if (e == cudaSuccess)
            e = launch_stitch(r->st, r->d_mean, de, step, norm, target, theta + (size_t)j * (r->B + 1),
                              r->d_joins, r->d_ok, r->B, r->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&oks[j], r->d_ok, sizeof(int), cudaMemcpyDeviceToHost, r->stream);
    }
    if (e == cudaSuccess) e = launch_jack(theta, r->m, r->B, d_err, r->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(err, d_err, (size_t)(r->B + 1) * 8, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    cudaFree(theta);
    cudaFree(d_err);
    if (e != cudaSuccess) return r->cuda_fail(e, "rewl_jackknife");
    for (int ok : oks)
        if (!ok) return r->fail(REWL_ERR_NOT_CONVERGED, "rewl_jackknife: a resample cannot be joined");
    return REWL_OK;
}

int rewl_windows_equal(int B, int h, double overlap, int *lo_hi)
{
    if (!lo_hi || B < 1 || h < 1) {
        g_err = "rewl_windows_equal: invalid argument";
        return REWL_ERR_INVALID_ARG;
    }
    std::vector<int> lo, hi;
    if (make_windows(B, h, overlap, lo, hi) != 0) {
        g_err = "rewl_windows_equal: windows do not overlap (too many windows or bad overlap)";
        return REWL_ERR_INVALID_ARG;
    }
    for (int w = 0; w < h; ++w) {
        lo_hi[w] = lo[w];
        lo_hi[h + w] = hi[w];
    }
    return REWL_OK;
}

int rewl_windows_late_balanced(const int *lo_hi, int h, const double *rounds_per_iter, int B,
                               int h_new, double overlap, int *lo_hi_out)
{
    if (!lo_hi || !rounds_per_iter || !lo_hi_out || h < 1 || B < 1 || h_new < 1) {
        g_err = "rewl_windows_late_balanced: invalid argument";
        return REWL_ERR_INVALID_ARG;
    }
    // per window a = (rounds per late iteration) / width^2; a bin costs sqrt(a) (the mean over
    // the windows covering it), so windows of equal summed cost have equal a * width^2
    std::vector<double> a(h, -1.0);
    double amax = 0.0;
    for (int w = 0; w < h; ++w) {
        const int lo = lo_hi[w], hi = lo_hi[h + w];
        if (lo < 0 || hi > B || hi < lo) {
            g_err = "rewl_windows_late_balanced: window outside [0, B]";
            return REWL_ERR_INVALID_ARG;
        }
        const double t = rounds_per_iter[w], wd = (double)(hi - lo + 1);
        if (t > 0.0 && std::isfinite(t)) {
            a[w] = t / (wd * wd);
            amax = std::max(amax, a[w]);
        }
    }
    if (!(amax > 0.0)) {
        g_err = "rewl_windows_late_balanced: no window has a measured iteration time";
        return REWL_ERR_INVALID_ARG;
    }
    std::vector<double> cost(B + 1, 0.0), cnt(B + 1, 0.0);
    for (int w = 0; w < h; ++w) {
        const double c = std::sqrt(a[w] > 0.0 ? a[w] : amax); // unmeasured: as the slowest
        for (int b = lo_hi[w]; b <= lo_hi[h + w]; ++b) {
            cost[b] += c;
            cnt[b] += 1.0;
        }
    }
    for (int b = 0; b <= B; ++b) cost[b] = cnt[b] > 0.0 ? cost[b] / cnt[b] : std::sqrt(amax);
    return rewl_windows_balanced(cost.data(), B, h_new, overlap, lo_hi_out);
}

int rewl_windows_balanced(const double *cost, int B, int h, double overlap, int *lo_hi)
{
    if (!cost || !lo_hi || B < 1 || h < 1 || !(overlap >= 0.0 && overlap < 1.0)) {
        g_err = "rewl_windows_balanced: invalid argument";
        return REWL_ERR_INVALID_ARG;
    }
    // cumulative cost C(b) = sum_{x < b} cost[x] + (cost of b)/2, then equal-size windows with
    // overlap o in the coordinate u = C / C_total (Fig. 1b: run-time balanced subdivision)
    std::vector<double> cum(B + 2, 0.0);
    for (int b = 0; b <= B; ++b) {
        if (!(cost[b] >= 0.0) || !std::isfinite(cost[b])) {
            g_err = "rewl_windows_balanced: cost must be finite and >= 0";
            return REWL_ERR_INVALID_ARG;
        }
        cum[b + 1] = cum[b] + cost[b];
    }
    const double tot = cum[B + 1];
    std::vector<int> lo(h), hi(h);
    if (h == 1 || !(tot > 0.0)) {
        if (make_windows(B, h, overlap, lo, hi) != 0) {
            g_err = "rewl_windows_balanced: windows do not overlap";
            return REWL_ERR_INVALID_ARG;
        }
    } else {
        const double W = 1.0 / (1.0 + (double)(h - 1) * (1.0 - overlap));
        const double st = (1.0 - overlap) * W;
        auto bin_at = [&](double u) { // first bin whose cumulative cost reaches u * tot
            const double target = u * tot;
            int a = 0, z = B;
            while (a < z) {
                const int mid = (a + z) / 2;
                if (cum[mid + 1] >= target) z = mid;
                else a = mid + 1;
            }
            return a;
        };
        for (int k = 0; k < h; ++k) {
            lo[k] = k == 0 ? 0 : bin_at((double)k * st);
            hi[k] = k == h - 1 ? B : bin_at((double)k * st + W);
        }
        // keep every window at least 5 bins wide and strictly overlapping its successor
        for (int k = 0; k < h; ++k) {
            if (k > 0 && lo[k] <= lo[k - 1]) lo[k] = lo[k - 1] + 1;
            if (hi[k] < lo[k] + 4) hi[k] = std::min(B, lo[k] + 4);
            if (k > 0 && hi[k] <= hi[k - 1]) hi[k] = std::min(B, hi[k - 1] + 1);
        }
        hi[h - 1] = B;
        for (int k = 0; k + 1 < h; ++k)
            if (lo[k + 1] > hi[k] - 1) lo[k + 1] = std::max(lo[k] + 1, hi[k] - 1);
        if (check_windows(B, lo, hi) != 0) {
            g_err = "rewl_windows_balanced: too many windows for this cost profile";
            return REWL_ERR_INVALID_ARG;
        }
    }
    for (int k = 0; k < h; ++k) {
        lo_hi[k] = lo[k];
        lo_hi[h + k] = hi[k];
    }
    return REWL_OK;
}

// per-bin first-iteration cost density of a run: mean over the windows covering the bin of
// (first-iteration rounds) / (window width)
static int prerun_cost(rewl_t pre, std::vector<double> &c)
{
    std::vector<long long> t1((size_t)pre->h);
    int rc = rewl_get_state(pre, "first_iter_round", t1.data(), t1.size() * 8);
    if (rc != REWL_OK) return rc;
    for (long long v : t1)
        if (v <= 0) return pre->fail(REWL_ERR_STATE, "pre-run: a window has not finished its first iteration");
    std::vector<double> n((size_t)pre->B + 1, 0.0);
    c.assign((size_t)pre->B + 1, 0.0);
    for (int w = 0; w < pre->h; ++w) {
        const double d = (double)t1[w] / (double)(pre->hi[w] - pre->lo[w] + 1);
        for (int b = pre->lo[w]; b <= pre->hi[w]; ++b) {
            c[b] += d;
            n[b] += 1.0;
        }
    }
    for (int b = 0; b <= pre->B; ++b) c[b] = n[b] > 0 ? c[b] / n[b] : 0.0;
    return REWL_OK;
}

int rewl_balanced_from_prerun(rewl_t pre, int h, double overlap, int *lo_hi)
{
    if (!pre || !lo_hi || h < 1) return REWL_ERR_INVALID_ARG;
    std::vector<double> c;
    int rc = prerun_cost(pre, c);
    if (rc != REWL_OK) return rc;
    rc = rewl_windows_balanced(c.data(), pre->B, h, overlap, lo_hi);
    if (rc != REWL_OK) return pre->fail(rc, g_err);
    return REWL_OK;
}

int rewl_balanced_scaled(rewl_t pre, int L, int h, double overlap, int *lo_hi)
{
    if (!pre || !lo_hi || h < 1 || L < 2) return REWL_ERR_INVALID_ARG;
    std::vector<double> c;
    int rc = prerun_cost(pre, c);
    if (rc != REWL_OK) return rc;
    // the same model on an L x L lattice: bins map through e = E/N (energy per site)
    const int N = L * L, B = pre->model == 0 ? N : 2 * N;
    std::vector<double> cs((size_t)B + 1);
    for (int b = 0; b <= B; ++b) {
        const double frac = (double)b / (double)B; // e = -2 + (2 or 1) * b/N, linear in b/B
        const int bp = (int)std::lround(frac * (double)pre->B);
        cs[b] = c[(size_t)std::min(std::max(bp, 0), pre->B)];
    }
    rc = rewl_windows_balanced(cs.data(), B, h, overlap, lo_hi);
    if (rc != REWL_OK) return pre->fail(rc, g_err);
    return REWL_OK;
}

int rewl_dims(rewl_t r, int *out)
{
    if (!r || !out) return REWL_ERR_INVALID_ARG;
    out[0] = r->N;
    out[1] = r->B;
    out[2] = r->h;
    out[3] = r->m;
    out[4] = r->W;
    out[5] = r->q;
    out[6] = r->L;
    out[7] = r->model;
    return REWL_OK;
}

int rewl_get_lng(rewl_t r, int window, int walker, double *out, int cap, int *lo, int *hi)
{
    if (!r || !out || window < 0 || window >= r->h || walker < -1 || walker >= r->m)
        return REWL_ERR_INVALID_ARG;
    const int nb = r->hi[window] - r->lo[window] + 1;
    if (cap < nb) return r->fail(REWL_ERR_BUFFER_TOO_SMALL, "rewl_get_lng: cap < window width");
    cudaError_t e;
    const double *src;
    if (walker < 0) {
        e = launch_window_mean(r->st, r->d_mean, r->stream);
        if (e != cudaSuccess) return r->cuda_fail(e, "window mean");
        src = r->d_mean + (size_t)window * r->W;
    } else {
        src = r->st.lng + ((size_t)window * r->m + walker) * r->W;
    }
    e = cudaMemcpyAsync(out, src, (size_t)nb * 8, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return r->cuda_fail(e, "rewl_get_lng");
    if (lo) *lo = r->lo[window];
    if (hi) *hi = r->hi[window];
    return REWL_OK;
}

int rewl_stitch(rewl_t r, double *out, int cap, int norm, int *joins)
{
    if (!r || !out || (norm != 0 && norm != 1)) return REWL_ERR_INVALID_ARG;
    if (cap < r->B + 1) return r->fail(REWL_ERR_BUFFER_TOO_SMALL, "rewl_stitch: cap < B+1");
    const double de = r->model == 0 ? 4.0 : 1.0;
    const int step = (r->model != 0 && r->q == 2) ? 2 : 1;
    const double target = norm == 0 ? (double)r->N * std::log((double)r->q) : std::log((double)r->q);
    cudaError_t e = launch_window_mean(r->st, r->d_mean, r->stream);
    if (e == cudaSuccess)
        e = launch_stitch(r->st, r->d_mean, de, step, norm, target, r->d_out, r->d_joins, r->d_ok,
                          r->B, r->stream);
    int ok = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, r->d_out, (size_t)(r->B + 1) * 8, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ok, r->d_ok, sizeof(int), cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess && joins && r->h > 1)
        e = cudaMemcpyAsync(joins, r->d_joins, (size_t)(r->h - 1) * sizeof(int), cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return r->cuda_fail(e, "rewl_stitch");
    if (!ok) return r->fail(REWL_ERR_NOT_CONVERGED, "rewl_stitch: windows cannot be joined");
    return REWL_OK;
}

// field table for rewl_get_state / rewl_set_state
struct Field {
    void *dev;
    size_t bytes;
    bool writable;
};

static bool field(rewl_t r, const std::string &f, Field &out)
{
    State &s = r->st;
    const size_t nw = (size_t)r->nw, W = (size_t)r->W, h = (size_t)r->h;
    if (f == "k") out = {s.k, nw * 4, true};
    else if (f == "lng") out = {s.lng, nw * W * 8, true};
    else if (f == "H") out = {s.H, nw * W * 4, true};
    else if (f == "step") out = {s.step, nw * 8, true};
    else if (f == "acc") out = {s.acc, nw * 8, false};
    else if (f == "flat") out = {s.flat, nw, true};
    else if (f == "lnf") out = {s.lnf, h * 8, true};
    else if (f == "iter") out = {s.iter, h * 4, true};
    else if (f == "finished") out = {s.finished, h, true};
    else if (f == "mask") out = {s.mask, h * W, true};
    else if (f == "swap_att") out = {s.swap_att, h * 8, false};
    else if (f == "swap_acc") out = {s.swap_acc, h * 8, false};
    else if (f == "pstep") out = {s.pstep, nw * 8, false};
    else if (f == "prep_restarts") out = {s.restarts, nw * 4, false};
    else if (f == "first_iter_round") out = {s.it1_round, h * 8, false};
    else if (f == "mode") out = {s.mode, h, true};
    else if (f == "frag") out = {s.frag, nw * W * 8, false};
    else if (f == "lo") out = {r->d_lohi, h * 4, false};
    else if (f == "hi") out = {r->d_lohi + h, h * 4, false};
    else return false;
    return true;
}

int rewl_get_state(rewl_t r, const char *name, void *out, size_t bytes)
{
    if (!r || !name || !out) return REWL_ERR_INVALID_ARG;
    const std::string f(name);
    cudaError_t e = cudaSuccess;
    if (f == "spins") { // gather per slot through the slot -> configuration map
        const size_t N = (size_t)r->N, nw = (size_t)r->nw;
        if (bytes != nw * N) return r->fail(REWL_ERR_BUFFER_TOO_SMALL, "spins: bytes mismatch");
        std::vector<int> cfg(nw);
        std::vector<int8_t> all(nw * (size_t)r->st.spin_stride);
        e = cudaMemcpyAsync(cfg.data(), r->st.cfg, nw * 4, cudaMemcpyDeviceToHost, r->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(all.data(), r->st.spins, all.size(), cudaMemcpyDeviceToHost, r->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
        if (e != cudaSuccess) return r->cuda_fail(e, "get spins");
        for (size_t i = 0; i < nw; ++i)
            std::memcpy((int8_t *)out + i * N, all.data() + (size_t)cfg[i] * r->st.spin_stride, N);
        return REWL_OK;
    }
    if (f == "lng_mean") { // window means (Sec. 2 average, walker order), [h][W]
        const size_t nbytes = (size_t)r->h * r->W * 8;
        if (bytes != nbytes) return r->fail(REWL_ERR_BUFFER_TOO_SMALL, "lng_mean: bytes mismatch");
        e = launch_window_mean(r->st, r->d_mean, r->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, r->d_mean, nbytes, cudaMemcpyDeviceToHost, r->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
        if (e != cudaSuccess) return r->cuda_fail(e, "lng_mean");
        return REWL_OK;
    }
    if (f == "round" || f == "n_exact" || f == "n_mismatch") {
        if (bytes != 8) return r->fail(REWL_ERR_BUFFER_TOO_SMALL, f + ": bytes must be 8");
        int rc = sync_status(r);
        if (rc != REWL_OK) return rc;
        if (f == "round") *(long long *)out = r->h_status->round;
        else if (f == "n_exact") *(unsigned long long *)out = r->h_status->n_exact;
        else *(unsigned long long *)out = r->h_status->n_mismatch;
        return REWL_OK;
    }
    Field fd;
    if (!field(r, f, fd)) return r->fail(REWL_ERR_INVALID_ARG, "unknown field " + f);
    if (bytes != fd.bytes) return r->fail(REWL_ERR_BUFFER_TOO_SMALL, f + ": bytes mismatch");
    e = cudaMemcpyAsync(out, fd.dev, bytes, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return r->cuda_fail(e, "rewl_get_state");
    return REWL_OK;
}

int rewl_set_state(rewl_t r, const char *name, const void *in, size_t bytes)
{
    if (!r || !name || !in) return REWL_ERR_INVALID_ARG;
    if (!r->inited) return r->fail(REWL_ERR_STATE, "rewl_set_state before rewl_init");
    const std::string f(name);
    cudaError_t e = cudaSuccess;
    if (f == "spins") { // write per slot through the map
        const size_t N = (size_t)r->N, nw = (size_t)r->nw;
        if (bytes != nw * N) return r->fail(REWL_ERR_BUFFER_TOO_SMALL, "spins: bytes mismatch");
        std::vector<int> cfg(nw);
        e = cudaMemcpyAsync(cfg.data(), r->st.cfg, nw * 4, cudaMemcpyDeviceToHost, r->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
        for (size_t i = 0; i < nw && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(r->st.spins + (size_t)cfg[i] * r->st.spin_stride,
                                (const int8_t *)in + i * N, N, cudaMemcpyHostToDevice, r->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
        if (e != cudaSuccess) return r->cuda_fail(e, "set spins");
        return REWL_OK;
    }
    if (f == "round") {
        if (bytes != 8) return r->fail(REWL_ERR_BUFFER_TOO_SMALL, "round: bytes must be 8");
        if (*(const long long *)in < 0) return r->fail(REWL_ERR_INVALID_ARG, "round: negative");
        e = cudaMemcpyAsync(&r->st.status->round, in, 8, cudaMemcpyHostToDevice, r->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
        if (e != cudaSuccess) return r->cuda_fail(e, "rewl_set_state(round)");
        return REWL_OK;
    }
    Field fd;
    if (!field(r, f, fd) || !fd.writable) return r->fail(REWL_ERR_INVALID_ARG, "field not writable: " + f);
    if (bytes != fd.bytes) return r->fail(REWL_ERR_BUFFER_TOO_SMALL, f + ": bytes mismatch");
    // values the kernels rely on
    if (f == "flat" || f == "finished" || f == "mask" || f == "mode") {
        for (size_t i = 0; i < bytes; ++i)
            if (((const uint8_t *)in)[i] > 1) return r->fail(REWL_ERR_INVALID_ARG, f + ": values must be 0 or 1");
    } else if (f == "lnf") {
        for (size_t i = 0; i < bytes / 8; ++i) {
            const double v = ((const double *)in)[i];
            if (!(v >= 0.0 && v < 0x1p20)) return r->fail(REWL_ERR_INVALID_ARG, "lnf: values must lie in [0, 2^20)");
        }
    } else if (f == "iter") {
        for (size_t i = 0; i < bytes / 4; ++i)
            if (((const int *)in)[i] < 0) return r->fail(REWL_ERR_INVALID_ARG, "iter: negative");
    }
    e = cudaMemcpyAsync(fd.dev, in, bytes, cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess && f == "finished") e = launch_set_done(r->st, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return r->cuda_fail(e, "rewl_set_state");
    return REWL_OK;
}

int rewl_stats(rewl_t r, rewl_stats_t *o)
{
    if (!r || !o) return REWL_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    const size_t nw = (size_t)r->nw, h = (size_t)r->h;
    std::vector<unsigned long long> step(nw), acc(nw), sa(h), sc(h);
    std::vector<int> rs(nw), iter(h);
    std::vector<double> lnf(h);
    std::vector<uint8_t> fin(h);
    int rc = REWL_OK;
    if ((rc = rewl_get_state(r, "step", step.data(), nw * 8))) return rc;
    if ((rc = rewl_get_state(r, "acc", acc.data(), nw * 8))) return rc;
    if ((rc = rewl_get_state(r, "swap_att", sa.data(), h * 8))) return rc;
    if ((rc = rewl_get_state(r, "swap_acc", sc.data(), h * 8))) return rc;
    if ((rc = rewl_get_state(r, "prep_restarts", rs.data(), nw * 4))) return rc;
    if ((rc = rewl_get_state(r, "iter", iter.data(), h * 4))) return rc;
    if ((rc = rewl_get_state(r, "lnf", lnf.data(), h * 8))) return rc;
    if ((rc = rewl_get_state(r, "finished", fin.data(), h))) return rc;
    if ((rc = sync_status(r))) return rc;
    o->rounds = r->h_status->round;
    o->exact_decisions = (long long)r->h_status->n_exact;
    for (size_t i = 0; i < nw; ++i) {
        o->attempts += (long long)step[i];
        o->accepted += (long long)acc[i];
        o->prep_restarts += rs[i];
    }
    o->min_iteration = 1 << 30;
    for (size_t w = 0; w < h; ++w) {
        o->swap_attempts += (long long)sa[w];
        o->swap_accepted += (long long)sc[w];
        o->windows_finished += fin[w];
        o->min_iteration = std::min(o->min_iteration, iter[w]);
        o->max_lnf = std::max(o->max_lnf, lnf[w]);
    }
    o->seconds = r->seconds;
    return REWL_OK;
}

// ---- checkpoints: header + the raw device arrays, in a fixed order
static const char CKPT_MAGIC[8] = {'R', 'E', 'W', 'L', 'C', 'K', '0', '2'};
struct CkptHeader {
    char magic[8];
    int model, L, h, m, W, N, spin_stride;
    long long interval;
    double lnf_final, flatness;
    uint64_t seed;
    uint32_t inst;
    int schedule;   // ln f schedule (must match the handle's)
    int production; // production mode of the run (restored)
    int has_hem;    // the (E, M) histogram follows the fields (restored)
};

static std::vector<Field> ckpt_fields(rewl_t r)
{
    State &s = r->st;
    const size_t nw = (size_t)r->nw, W = (size_t)r->W, h = (size_t)r->h;
    return {{s.spins, nw * s.spin_stride, true}, {s.cfg, nw * 4, true}, {s.k, nw * 4, true},
            {s.lng, nw * W * 8, true},          {s.H, nw * W * 4, true}, {s.step, nw * 8, true},
            {s.acc, nw * 8, true},              {s.pstep, nw * 8, true}, {s.restarts, nw * 4, true},
            {s.flat, nw, true},                 {r->d_lohi, 2 * h * 4, true}, {s.lnf, h * 8, true},
            {s.iter, h * 4, true},              {s.finished, h, true},   {s.mask, h * W, true},
            {s.swap_att, h * 8, true},          {s.swap_acc, h * 8, true}, {s.status, sizeof(DevStatus), true},
            {s.it1_round, h * 8, true},         {s.mode, h, true}, {s.frag, nw * W * 8, true}};
}

static size_t hem_bytes(rewl_t r) { return (size_t)r->h * r->W * ((size_t)r->N + 1) * 4u; }

int rewl_checkpoint(rewl_t r, const char *path)
{
    if (!r || !path) return REWL_ERR_INVALID_ARG;
    if (!r->inited) return r->fail(REWL_ERR_STATE, "rewl_checkpoint before rewl_init");
    CkptHeader hd{};
    std::memcpy(hd.magic, CKPT_MAGIC, 8);
    hd.model = r->model; hd.L = r->L; hd.h = r->h; hd.m = r->m; hd.W = r->W; hd.N = r->N;
    hd.spin_stride = r->st.spin_stride; hd.interval = r->interval; hd.lnf_final = r->lnf_final;
    hd.flatness = r->flatness; hd.seed = r->seed; hd.inst = r->inst;
    hd.schedule = r->schedule; hd.production = r->production; hd.has_hem = r->st.hem != nullptr;
    std::vector<Field> fields = ckpt_fields(r);
    if (r->st.hem) fields.push_back({r->st.hem, hem_bytes(r), true});
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return r->fail(REWL_ERR_IO, std::string("cannot open ") + path);
    bool ok = std::fwrite(&hd, sizeof(hd), 1, fp) == 1;
    for (const Field &f : fields) {
        if (!ok) break;
        std::vector<unsigned char> buf(f.bytes);
        cudaError_t e = cudaMemcpyAsync(buf.data(), f.dev, f.bytes, cudaMemcpyDeviceToHost, r->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
        if (e != cudaSuccess) {
            std::fclose(fp);
            return r->cuda_fail(e, "checkpoint");
        }
        ok = std::fwrite(buf.data(), 1, f.bytes, fp) == f.bytes;
    }
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return r->fail(REWL_ERR_IO, std::string("write failed: ") + path);
    return REWL_OK;
}

int rewl_restore(rewl_t r, const char *path)
{
    if (!r || !path) return REWL_ERR_INVALID_ARG;
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return r->fail(REWL_ERR_IO, std::string("cannot open ") + path);
    CkptHeader hd{};
    if (std::fread(&hd, sizeof(hd), 1, fp) != 1 || std::memcmp(hd.magic, CKPT_MAGIC, 8) != 0) {
        std::fclose(fp);
        return r->fail(REWL_ERR_IO, "not a REWL checkpoint");
    }
    if (hd.model != r->model || hd.L != r->L || hd.h != r->h || hd.m != r->m || hd.W != r->W ||
        hd.N != r->N || hd.spin_stride != r->st.spin_stride || hd.interval != r->interval ||
        hd.lnf_final != r->lnf_final || hd.flatness != r->flatness || hd.seed != r->seed ||
        hd.inst != r->inst || hd.schedule != r->schedule || (hd.production != 0 && hd.production != 1) ||
        (hd.has_hem != 0 && hd.has_hem != 1) || (hd.has_hem && r->model != 0)) {
        std::fclose(fp);
        return r->fail(REWL_ERR_INVALID_ARG, "checkpoint parameters differ from the handle's");
    }
    std::vector<Field> fields = ckpt_fields(r);
    std::vector<std::vector<unsigned char>> bufs;
    if (hd.has_hem) fields.push_back({nullptr, hem_bytes(r), true});
    for (const Field &f : fields) {
        bufs.emplace_back(f.bytes);
        if (std::fread(bufs.back().data(), 1, f.bytes, fp) != f.bytes) {
            std::fclose(fp);
            return r->fail(REWL_ERR_IO, "truncated checkpoint");
        }
    }
    std::fclose(fp);
    // window bounds must match the handle's layout
    std::vector<int> lohi(2 * r->h);
    std::memcpy(lohi.data(), bufs[10].data(), lohi.size() * 4);
    for (int w = 0; w < r->h; ++w)
        if (lohi[w] != r->lo[w] || lohi[r->h + w] != r->hi[w])
            return r->fail(REWL_ERR_INVALID_ARG, "checkpoint window layout differs");
    // run mode and (E, M) measurement as they were when the checkpoint was written (the
    // measurement exists for the Ising model only)
    if (r->model == 0) {
        const int rc = rewl_set_param(r, "measure_em", hd.has_hem ? 1.0 : 0.0);
        if (rc != REWL_OK) return rc;
    }
    if (hd.has_hem) fields.back().dev = r->st.hem;
    size_t i = 0;
    for (const Field &f : fields) {
        cudaError_t e = cudaMemcpyAsync(f.dev, bufs[i++].data(), f.bytes, cudaMemcpyHostToDevice, r->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
        if (e != cudaSuccess) return r->cuda_fail(e, "restore");
    }
    if (r->graph) cudaGraphExecDestroy(r->graph);
    r->graph = nullptr;
    r->production = hd.production;
    r->st.production = hd.production;
    r->st.schedule = r->schedule; // rewl_init, which a restore replaces, sets it otherwise
    r->inited = true;
    return REWL_OK;
}

void rewl_destroy(rewl_t r)
{
    if (!r) return;
    if (r->stream) cudaStreamSynchronize(r->stream);
    for (auto *v : {&r->ev_used, &r->ev_free})
        for (auto &ev : *v) {
            cudaEventDestroy(ev.first);
            cudaEventDestroy(ev.second);
        }
    release(r);
    delete r;
}

const char *rewl_last_error(rewl_t r)
{
    if (r) return r->err.c_str();
    return g_err.c_str();
}

// ---- replay through the production move kernel
int rewl_replay(int model, int L, int n, int W, int T, void *spins, void *k, const void *lo,
                const void *hi, void *lng, void *H, const void *lnf, const void *frozen,
                const void *words, void *acc, void *dk, void *stream)
{
    if (n < 0 || L < 2 || L > 255 || W < 1 || T < 1 || T > 100000000 || (model != 0 && (model < 2 || model > 127)) ||
        !spins || !k || !lo || !hi || !lng || !H || !lnf || !frozen || !words || !acc || !dk) {
        g_err = "rewl_replay: invalid argument";
        return REWL_ERR_INVALID_ARG;
    }
    if (n == 0) return REWL_OK;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    State s{};
    s.model = model;
    s.q = model == 0 ? 2 : model;
    s.L = L;
    s.N = L * L;
    s.nw = n;
    s.m = 1;
    s.h = n;
    s.W = W;
    s.spin_stride = s.N;
    s.vec_spins = (s.N & 15) == 0 && ((uintptr_t)spins & 15) == 0;
    s.magic = (uint32_t)((0x100000000ULL + (uint64_t)L - 1) / (uint64_t)L);
    for (uint32_t site = 0; site < (uint32_t)s.N; ++site)
        if ((uint32_t)(((uint64_t)site * s.magic) >> 32) != site / (uint32_t)L) {
            g_err = "rewl_replay: lattice too large";
            return REWL_ERR_INVALID_ARG;
        }
    if (move_smem_per_walker(s.N, W) > MAX_SMEM_PER_CTA) {
        g_err = "rewl_replay: lattice and window do not fit in shared memory";
        return REWL_ERR_INVALID_ARG;
    }
    s.spins = (int8_t *)spins;
    s.cfg = nullptr;
    s.k = (int *)k;
    s.lng = (double *)lng;
    s.H = (uint32_t *)H;
    s.lo = (const int *)lo;
    s.hi = (const int *)hi;
    s.lnf = (double *)lnf;
    s.finished = (uint8_t *)frozen;
    // scratch: allocated here, zeroed on the caller's stream so the kernel is ordered after it
    e = cudaMalloc(&s.step, (size_t)n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&s.acc, (size_t)n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&s.status, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemsetAsync(s.step, 0, (size_t)n * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.acc, 0, (size_t)n * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.status, 0, sizeof(DevStatus), st);
    if (e != cudaSuccess) {
        g_err = std::string("rewl_replay alloc: ") + cudaGetErrorString(e);
        cudaFree(s.step); cudaFree(s.acc); cudaFree(s.status);
        return REWL_ERR_CUDA;
    }
    MoveCfg c{};
    c.T = T;
    c.walkers_per_block = 4;
    while (c.walkers_per_block > 1 && (size_t)c.walkers_per_block * move_smem_per_walker(s.N, W) > MAX_SMEM_PER_CTA)
        c.walkers_per_block >>= 1;
    c.eps_l = LNU32_EPS;
    c.words = (const uint32_t *)words;
    c.acc_out = (int *)acc;
    c.dk_out = (int *)dk;
    e = launch_move(s, c, st);
    DevStatus hs{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, s.status, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(s.step);
    cudaFree(s.acc);
    cudaFree(s.status);
    if (e != cudaSuccess) {
        g_err = std::string("rewl_replay: ") + cudaGetErrorString(e);
        return REWL_ERR_CUDA;
    }
    if (hs.err) {
        g_err = (hs.err & ERR_INPUT) ? "rewl_replay: k outside [lo, hi] or window wider than W"
                                     : "rewl_replay: ln g or ln f out of the supported range";
        return REWL_ERR_INVALID_ARG;
    }
    return REWL_OK;
}

} // extern "C"

// ---- replay without allocation: the per-case scratch of the move kernel (step and
// acceptance counters, run status) lives in one fixed device array instead of cudaMalloc.
namespace {
struct ReplayScratch {
    unsigned long long step[REWL_REPLAY_STATIC_MAX_N];
    unsigned long long acc[REWL_REPLAY_STATIC_MAX_N];
    DevStatus status;
};
constexpr int SCRATCH_MAX_DEVICES = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[SCRATCH_MAX_DEVICES] = {};
} // namespace

// Every GPU that loads the library holds this array (about 256 KB) until the process exits.
static __device__ __align__(256) unsigned char g_replay_scratch[sizeof(ReplayScratch)];

// Device address of g_replay_scratch on the current device.  The first call on a device looks
// it up (cudaGetSymbolAddress, with that device current); later calls reuse the address.
static int replay_scratch(ReplayScratch **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        g_err = std::string("rewl_replay_static: cudaGetDevice: ") + cudaGetErrorString(e);
        return REWL_ERR_CUDA;
    }
    if (dev < 0 || dev >= SCRATCH_MAX_DEVICES) {
        g_err = "rewl_replay_static: device index out of range";
        return REWL_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_replay_scratch);
        if (e != cudaSuccess || !p) {
            g_err = std::string("rewl_replay_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return REWL_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<ReplayScratch *>(g_scratch_addr[dev]);
    return REWL_OK;
}

extern "C" {

int rewl_replay_static(int model, int L, int n, int W, int T, void *spins, void *k, const void *lo,
                       const void *hi, void *lng, void *H, const void *lnf, const void *frozen,
                       const void *words, void *acc, void *dk, void *stream)
{
    if (n < 0 || L < 2 || L > 255 || W < 1 || T < 1 || T > 100000000 || (model != 0 && (model < 2 || model > 127)) ||
        !spins || !k || !lo || !hi || !lng || !H || !lnf || !frozen || !words || !acc || !dk) {
        g_err = "rewl_replay_static: invalid argument";
        return REWL_ERR_INVALID_ARG;
    }
    if (n > REWL_REPLAY_STATIC_MAX_N) {
        g_err = "rewl_replay_static: n exceeds REWL_REPLAY_STATIC_MAX_N (" +
                std::to_string(REWL_REPLAY_STATIC_MAX_N) + ") cases";
        return REWL_ERR_INVALID_ARG;
    }
    if (n == 0) return REWL_OK;
    cudaStream_t st = (cudaStream_t)stream;
    State s{};
    s.model = model;
    s.q = model == 0 ? 2 : model;
    s.L = L;
    s.N = L * L;
    s.nw = n;
    s.m = 1;
    s.h = n;
    s.W = W;
    s.spin_stride = s.N;
    s.vec_spins = (s.N & 15) == 0 && ((uintptr_t)spins & 15) == 0;
    s.magic = (uint32_t)((0x100000000ULL + (uint64_t)L - 1) / (uint64_t)L);
    for (uint32_t site = 0; site < (uint32_t)s.N; ++site)
        if ((uint32_t)(((uint64_t)site * s.magic) >> 32) != site / (uint32_t)L) {
            g_err = "rewl_replay_static: lattice too large";
            return REWL_ERR_INVALID_ARG;
        }
    if (move_smem_per_walker(s.N, W) > MAX_SMEM_PER_CTA) {
        g_err = "rewl_replay_static: lattice and window do not fit in shared memory";
        return REWL_ERR_INVALID_ARG;
    }
    ReplayScratch *sc = nullptr;
    int rc = replay_scratch(&sc);
    if (rc != REWL_OK) return rc;
    s.spins = (int8_t *)spins;
    s.cfg = nullptr;
    s.k = (int *)k;
    s.lng = (double *)lng;
    s.H = (uint32_t *)H;
    s.lo = (const int *)lo;
    s.hi = (const int *)hi;
    s.lnf = (double *)lnf;
    s.finished = (uint8_t *)frozen;
    s.step = sc->step;
    s.acc = sc->acc;
    s.status = &sc->status;
    // the array keeps the previous call's contents: the counters and the status start at zero
    cudaError_t e = cudaMemsetAsync(sc->step, 0, (size_t)n * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->acc, 0, (size_t)n * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&sc->status, 0, sizeof(DevStatus), st);
    MoveCfg c{};
    c.T = T;
    c.walkers_per_block = 4;
    while (c.walkers_per_block > 1 && (size_t)c.walkers_per_block * move_smem_per_walker(s.N, W) > MAX_SMEM_PER_CTA)
        c.walkers_per_block >>= 1;
    c.eps_l = LNU32_EPS;
    c.words = (const uint32_t *)words;
    c.acc_out = (int *)acc;
    c.dk_out = (int *)dk;
    if (e == cudaSuccess) e = launch_move(s, c, st);
    DevStatus hs{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, &sc->status, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        g_err = std::string("rewl_replay_static: ") + cudaGetErrorString(e);
        return REWL_ERR_CUDA;
    }
    if (hs.err) {
        g_err = (hs.err & ERR_INPUT) ? "rewl_replay_static: k outside [lo, hi] or window wider than W"
                                     : "rewl_replay_static: ln g or ln f out of the supported range";
        return REWL_ERR_INVALID_ARG;
    }
    return REWL_OK;
}

int rewl_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n, void *stream)
{
    cudaError_t e = launch_philox(ctr, key, out, n, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        g_err = cudaGetErrorString(e);
        return REWL_ERR_CUDA;
    }
    return REWL_OK;
}

int rewl_lnu(const uint32_t *w, double *out, int n, void *stream)
{
    cudaError_t e = launch_lnu(w, out, n, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        g_err = cudaGetErrorString(e);
        return REWL_ERR_CUDA;
    }
    return REWL_OK;
}

int rewl_lnu_bound(uint64_t begin, uint64_t end, double *max_err, unsigned long long *n_bad, void *stream)
{
    if (end > (1ULL << 32) || !max_err || !n_bad) return REWL_ERR_INVALID_ARG;
    cudaError_t e = launch_lnu_bound(begin, end, max_err, n_bad, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        g_err = cudaGetErrorString(e);
        return REWL_ERR_CUDA;
    }
    return REWL_OK;
}

double rewl_lnu_eps(void) { return LNU32_EPS; }

int rewl_thermo(const double *lng, int model, int L, const double *T, int nT, double *U, double *C,
                void *stream)
{
    if (!lng || !T || !U || !C || nT < 0 || L < 2 || (model != 0 && model < 2)) {
        g_err = "rewl_thermo: invalid argument";
        return REWL_ERR_INVALID_ARG;
    }
    cudaError_t e = launch_thermo(lng, model, L, T, nT, U, C, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        g_err = cudaGetErrorString(e);
        return REWL_ERR_CUDA;
    }
    return REWL_OK;
}

int rewl_seqadd(const double *x, const double *f, const uint32_t *c, double *out, int n, void *stream)
{
    cudaError_t e = launch_seqadd(x, f, c, out, n, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        g_err = cudaGetErrorString(e);
        return REWL_ERR_CUDA;
    }
    return REWL_OK;
}

} // extern "C"
