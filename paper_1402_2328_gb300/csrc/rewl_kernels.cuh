// rewl_kernels.cuh -- kernel argument blocks and launchers shared by the host runtime.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace rewl {

// Device-side run status (one per handle).
struct DevStatus {
    long long round;              // rounds completed
    int done;                     // every window finished
    int err;                      // ERR_* bits
    unsigned long long n_exact;   // moves decided by the float64 path
    unsigned long long n_mismatch;// check_all: screen decisions that disagreed (must stay 0)
};
enum : int { ERR_PREP = 1, ERR_RANGE = 2, ERR_INPUT = 4 };
constexpr int MAX_M = 1024; // walkers per window (exchange permutation in shared memory)
constexpr size_t MAX_SMEM_PER_CTA = 227u * 1024u;

// Per-walker-slot state of one REWL instance, all device pointers.
struct State {
    int model, q, L, N, nw, m, h, W, spin_stride;
    int vec_spins;            // lattices 16-byte aligned with N % 16 == 0: int4 copies
    uint32_t magic;           // ceil(2^32 / L)
    int8_t *spins;            // [nw][spin_stride] lattices (owned by configuration index)
    int *cfg;                 // [nw] slot -> configuration index
    int *k;                   // [nw] current bin of the slot's configuration
    double *lng;              // [nw][W] window-local ln g
    uint32_t *H;              // [nw][W]
    unsigned long long *step; // [nw]
    unsigned long long *acc;  // [nw]
    unsigned long long *pstep;// [nw]
    int *restarts;            // [nw]
    uint8_t *flat;            // [nw]
    const int *lo, *hi;       // [h]
    double *lnf;              // [h]
    int *iter;                // [h]
    uint8_t *finished;        // [h]
    uint8_t *mask;            // [h][W]
    unsigned long long *swap_att, *swap_acc; // [h]
    long long *it1_round;     // [h] rounds done when the first iteration ended (0: not yet)
    uint8_t *mode;            // [h] 0: ln f halving, 1: ln f = 1/t
    int schedule;             // 0: halving only, 1: switch to 1/t
    double *frag;             // [nw][W] ln g of each walker just before its window's last average
    uint32_t *hem;            // [h][W][N+1] (bin, up spins) counts, nullptr: not measured
    int production;           // rounds continue after every window finished
    DevStatus *status;
    uint32_t key0, key1, inst;
    int w0, slot0;            // window-sharded run: global index of window 0 / walker slot 0
};

struct MoveCfg {
    int T;                  // attempts per walker in this launch
    int walkers_per_block;  // walkers per CTA (warps, or threads with layout 1)
    int layout;             // 0: one warp per walker, 1: one thread per walker
    int check_all;
    double eps_l;
    const uint32_t *words;  // replay: [nw][T][3], else nullptr (Philox)
    int *acc_out, *dk_out;  // replay: [nw][T]
};

// 32-bit words of the per-walker visited-bin bit set (padded to 16 bytes)
__host__ __device__ inline int visw(int W) { return (((W + 31) >> 5) + 3) & ~3; }

// Shared memory of one walker in the move kernel: lattice (16-byte padded), int64 ln g
// shadow over the window (padded to 4 bins; the visit counts are recovered from it), the
// visited-bin bit set, uint16 claim stamps per site.
__host__ __device__ inline size_t move_smem_per_walker(int N, int W)
{
    return (size_t)((N + 15) & ~15) + (size_t)((W + 3) & ~3) * 8u + (size_t)visw(W) * 4u +
           (size_t)((N + 7) & ~7) * 2u;
}
// Shared memory of one walker of the thread-per-walker layout: lattice (16-byte padded) and the
// int64 ln g shadow over the window (padded to 2 bins, 16 bytes).
__host__ __device__ inline size_t move_smem_per_thread_walker(int N, int W)
{
    return (size_t)((N + 15) & ~15) + (size_t)((W + 1) & ~1) * 8u;
}
cudaError_t launch_move(const State &s, const MoveCfg &c, cudaStream_t st);
// Batched instances: states/jobs/tables are device arrays (see the kernels).
cudaError_t launch_move_batch(const State *states, const int4 *jobs, int njobs, int walkers_per_block,
                              size_t smem, const MoveCfg &c, cudaStream_t st);
cudaError_t launch_check_batch(const State *states, const int2 *tab, int n, const double2 *prm,
                               cudaStream_t st);
cudaError_t launch_swap_batch(const State *states, const int2 *tab, int n, cudaStream_t st);
cudaError_t launch_round_end_batch(const State *states, int n, cudaStream_t st);
cudaError_t launch_init_prep(const State &s, long long prep_budget, cudaStream_t st);
cudaError_t launch_check(const State &s, double flatness, double lnf_final, cudaStream_t st);
cudaError_t launch_swap(const State &s, cudaStream_t st);
cudaError_t launch_round_end(const State &s, cudaStream_t st);
cudaError_t launch_set_done(const State &s, cudaStream_t st);
// joint density of states g(E, M) (rewl_em.cu)
cudaError_t launch_measure_em(const State &s, cudaStream_t st);
cudaError_t launch_window_mean(const State &s, double *out /*[h][W]*/, cudaStream_t st);
cudaError_t launch_stitch(const State &s, const double *mean, double de, int step, int norm,
                          double target, double *out /*B+1*/, int *joins /*h-1*/,
                          int *ok /*1*/, int B, cudaStream_t st);

// window-sharded runs: the exchange of the pair across a shard boundary (Eq. 1), in four steps
// (side 1: this shard holds the pair's lower window, its last; side 0: the upper, its first)
cudaError_t launch_bnd_bins(const State &s, int side, int *bins, cudaStream_t st);
cudaError_t launch_bnd_half(const State &s, int side, int plo, int phi, const int *pbins,
                            double *half, cudaStream_t st);
cudaError_t launch_bnd_decide(const State &s, int side, const double *half, const double *phalf,
                              uint8_t *acc, int8_t *lat_out, cudaStream_t st);
cudaError_t launch_bnd_import(const State &s, int side, const int *pbins, const uint8_t *acc,
                              const int8_t *plat, cudaStream_t st);
cudaError_t launch_loo_mean(const State &s, int j, double *out /*[h][W]*/, cudaStream_t st);
cudaError_t launch_jack(const double *theta /*[m][B+1]*/, int m, int B, double *err, cudaStream_t st);
cudaError_t launch_thermo(const double *lng, int model, int L, const double *T, int nT, double *U,
                          double *C, cudaStream_t st);
cudaError_t launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n,
                          cudaStream_t st);
cudaError_t launch_lnu(const uint32_t *w, double *out, int n, cudaStream_t st);
cudaError_t launch_lnu_bound(uint64_t begin, uint64_t end, double *max_err,
                             unsigned long long *n_bad, cudaStream_t st);
cudaError_t launch_seqadd(const double *x, const double *f, const uint32_t *c, double *out,
                          int n, cudaStream_t st);

} // namespace rewl
