// rewl_handle.h -- private: the single-instance handle shared by the host runtime files.
#pragma once
#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "rewl.h"
#include "rewl_kernels.cuh"

extern thread_local std::string g_err;

struct rewl_s {
    // parameters
    int model = 0, q = 2, L = 0, N = 0, B = 0, h = 0, m = 0, nw = 0, W = 0;
    double overlap = 0.75, lnf_final = 1e-8, flatness = 0.8, lnf_init = 1.0;
    uint64_t seed = 0;
    uint32_t inst = 0;
    long long interval = 10000, prep_budget = 100;
    int graph_rounds = 32, wpb = 0, check_all = 0, profile = 0, schedule = 0, production = 0;
    int layout = 0; // move kernel: 0 one warp per walker, 1 one thread per walker
    // window-sharded run: global index of this handle's first window, and the bins of the
    // neighbouring shards' boundary windows (lo, hi of window w_begin-1, then of w_end; -1: none)
    int shard = 0, w_begin = 0;
    int nbr[4] = {-1, -1, -1, -1};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used, ev_free; // move-kernel timing
    std::vector<int> lo, hi;
    std::vector<double> lng_init;
    bool inited = false, allocated = false;
    cudaStream_t stream = nullptr;
    // device state
    rewl::State st{};
    int *d_lohi = nullptr;
    double *d_mean = nullptr, *d_out = nullptr;
    int *d_joins = nullptr, *d_ok = nullptr;
    rewl::DevStatus *h_status = nullptr; // pinned
    // graphs
    cudaGraphExec_t graph = nullptr;
    int graph_len = 0;
    // bookkeeping
    std::string err;
    double seconds = 0.0;
    std::atomic<int> abort_flag{0};
    int sms = 148;

    int fail(int code, const std::string &msg)
    {
        err = msg;
        g_err = msg;
        return code;
    }
    int cuda_fail(cudaError_t e, const char *where)
    {
        return fail(REWL_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    }
};


// enqueue one round of the single-instance path on r->stream (rewl_host.cu)
extern "C" cudaError_t rewl_enqueue_round(rewl_t r);
