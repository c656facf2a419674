// rewl_em.cu -- joint density of states g(E, M) of the Ising model (Sec. 3, Eqs. 3-4).
//
// 1. measurement: after the moves of every round each walker's (bin k, up spins j) is counted
//    in its window's histogram H_w(k, j) (M = 2j - N).  Rounds after every window finished run
//    on in production mode: ln g is frozen, so each window performs a multicanonical walk with
//    weight 1/g_w(E) and P_w(M | E) = g(E, M) / g(E).
// 2. fragments: S_w(k, j) = mean ln g_w(k) + ln H_w(k, j) - ln sum_j H_w(k, j).
// 3. joining (Eq. 3): for adjacent windows the point of the overlap where the unit normals
//    (dS/dE, dS/dM, -1) agree best (largest dot product; ties: smallest k, then j) fixes the
//    shift of window w+1; Eq. (4) merges the windows in order, g = (g_i + g_j) / 2 where both
//    are present; the result is normalised to sum g = 2^N.
// Every decision (the join points) is taken with the same float64 operations, in the same
// order, as the plain implementation the tests compare with; logarithms of counts use the
// reproducible ln64 of rewl_device.cuh.

#include <algorithm>
#include <climits>
#include <cmath>
#include <string>
#include <vector>

#include "rewl_device.cuh"
#include "rewl_handle.h"

using namespace rewl;

namespace {

constexpr int EM_THREADS = 256;
constexpr double EM_LN2 = 0x1.62e42fefa39efp-1;

__global__ void k_measure_em(State s)
{
    if (s.status->done) return;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= s.nw) return; // uniform per warp
    const int8_t *sp = s.spins + (size_t)s.cfg[warp] * s.spin_stride;
    unsigned up = 0;
    for (int i = lane; i < s.N; i += 32) up += sp[i] > 0 ? 1u : 0u;
    up = __reduce_add_sync(0xffffffffu, up);
    if (lane == 0) {
        const int w = warp / s.m;
        atomicAdd(&s.hem[((size_t)w * s.W + (size_t)(s.k[warp] - s.lo[w])) * (size_t)(s.N + 1) + up], 1u);
    }
}

__device__ unsigned long long block_sum_u64(unsigned long long v)
{
    __shared__ unsigned long long part[EM_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0;
    for (int i = 0; i < EM_THREADS / 32; ++i) t += part[i];
    __syncthreads();
    return t;
}

// one block per (window, row): S[w][b][j] = (mean + ln H) - ln sum_j H, -inf where absent
__global__ void k_frag_em(State s, const double *__restrict__ mean, double *__restrict__ S)
{
    const int w = blockIdx.x / s.W, b = blockIdx.x % s.W, N1 = s.N + 1;
    const uint32_t *row = s.hem + ((size_t)w * s.W + b) * N1;
    unsigned long long t = 0;
    for (int j = threadIdx.x; j < N1; j += blockDim.x) t += row[j];
    const unsigned long long tot = block_sum_u64(t);
    const bool ok = b <= s.hi[w] - s.lo[w] && s.mask[(size_t)w * s.W + b] && tot > 0;
    const double lt = ok ? ln64((double)tot) : 0.0;
    const double mv = mean[(size_t)w * s.W + b];
    double *out = S + ((size_t)w * s.W + b) * N1;
    for (int j = threadIdx.x; j < N1; j += blockDim.x)
        out[j] = (ok && row[j] > 0u) ? __dsub_rn(__dadd_rn(mv, ln64((double)row[j])), lt) : -INFINITY;
}

// derivative along one axis at index i of n points with stride st: 5-point stencil where the
// four neighbours are present, else 3-point, else none
__device__ bool em_deriv(const double *S, int i, int n, size_t st, double d, double *out)
{
    if (i - 2 >= 0 && i + 2 < n && S[(i - 2) * st] > -INFINITY && S[(i - 1) * st] > -INFINITY &&
        S[(i + 1) * st] > -INFINITY && S[(i + 2) * st] > -INFINITY) {
        const double num = __dadd_rn(__dsub_rn(__dadd_rn(-S[(i + 2) * st], __dmul_rn(8.0, S[(i + 1) * st])),
                                               __dmul_rn(8.0, S[(i - 1) * st])),
                                     S[(i - 2) * st]);
        *out = __ddiv_rn(num, __dmul_rn(12.0, d));
        return true;
    }
    if (i - 1 >= 0 && i + 1 < n && S[(i - 1) * st] > -INFINITY && S[(i + 1) * st] > -INFINITY) {
        *out = __ddiv_rn(__dsub_rn(S[(i + 1) * st], S[(i - 1) * st]), __dmul_rn(2.0, d));
        return true;
    }
    return false;
}

__device__ bool em_grad(const double *Sw, int nb, int N1, int b, int j, double de, double dq,
                        double *gE, double *gQ)
{
    return em_deriv(Sw + j, b, nb, (size_t)N1, de, gE) && em_deriv(Sw + (size_t)b * N1, j, N1, 1, dq, gQ);
}

struct Best {
    double dot;
    long long t, fb; // argmax index (ties: smaller), fallback key (smaller wins)
};

__device__ Best better(Best a, Best b)
{
    Best r = a;
    if (b.dot > a.dot || (b.dot == a.dot && b.t < a.t)) {
        r.dot = b.dot;
        r.t = b.t;
    }
    r.fb = a.fb < b.fb ? a.fb : b.fb;
    return r;
}

// grid (blocks, h-1): candidates of pair (p, p+1), one partial result per block
__global__ void k_join_cand(const double *__restrict__ S, const int *__restrict__ lo,
                            const int *__restrict__ hi, int W, int N1, double de, double dq,
                            Best *__restrict__ part)
{
    const int p = blockIdx.y;
    const int k0 = lo[p + 1];
    const long long npts = (long long)(hi[p] - k0 + 1) * N1;
    const double *Sa = S + (size_t)p * W * N1, *Sb = S + (size_t)(p + 1) * W * N1;
    const int nba = hi[p] - lo[p] + 1, nbb = hi[p + 1] - lo[p + 1] + 1, mid2 = lo[p + 1] + hi[p];
    Best best{-INFINITY, LLONG_MAX, LLONG_MAX};
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < npts;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = k0 + (int)(t / N1), j = (int)(t % N1);
        const int a = k - lo[p], b = k - lo[p + 1];
        if (!(Sa[(size_t)a * N1 + j] > -INFINITY && Sb[(size_t)b * N1 + j] > -INFINITY)) continue;
        const long long d = (long long)abs(2 * k - mid2);
        const long long f = d * npts + t;
        if (f < best.fb) best.fb = f;
        double aE, aQ, bE, bQ;
        if (!em_grad(Sa, nba, N1, a, j, de, dq, &aE, &aQ)) continue;
        if (!em_grad(Sb, nbb, N1, b, j, de, dq, &bE, &bQ)) continue;
        const double num = __dadd_rn(__dadd_rn(__dmul_rn(aE, bE), __dmul_rn(aQ, bQ)), 1.0);
        const double den = __dmul_rn(__dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(aE, aE), __dmul_rn(aQ, aQ)), 1.0)),
                                     __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(bE, bE), __dmul_rn(bQ, bQ)), 1.0)));
        const double dot = __ddiv_rn(num, den);
        if (dot > best.dot || (dot == best.dot && t < best.t)) {
            best.dot = dot;
            best.t = t;
        }
    }
    __shared__ Best sh[EM_THREADS];
    sh[threadIdx.x] = best;
    __syncthreads();
    for (int o = EM_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] = better(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)p * gridDim.x + blockIdx.x] = sh[0];
}

// one thread: join points and the chain of shifts (shift of window w+1 from the already
// shifted window w)
__global__ void k_join_finish(const double *__restrict__ S, const int *__restrict__ lo,
                              const int *__restrict__ hi, int h, int W, int N1, int nblk,
                              const Best *__restrict__ part, double *shift, int *joins, int *ok)
{
    shift[0] = 0.0;
    *ok = 0;
    for (int p = 0; p + 1 < h; ++p) {
        Best b{-INFINITY, LLONG_MAX, LLONG_MAX};
        for (int i = 0; i < nblk; ++i) b = better(b, part[(size_t)p * nblk + i]);
        const long long npts = (long long)(hi[p] - lo[p + 1] + 1) * N1;
        long long t;
        if (b.t != LLONG_MAX) t = b.t;
        else if (b.fb != LLONG_MAX) t = b.fb % npts;
        else return;
        const int k = lo[p + 1] + (int)(t / N1), j = (int)(t % N1);
        const double va = S[((size_t)p * W + (k - lo[p])) * N1 + j];
        const double vb = S[((size_t)(p + 1) * W + (k - lo[p + 1])) * N1 + j];
        shift[p + 1] = __dsub_rn(__dadd_rn(va, shift[p]), vb);
        joins[2 * p] = k;
        joins[2 * p + 1] = j;
    }
    *ok = 1;
}

// Eq. (4), windows merged in order at every point
__global__ void k_combine_em(const double *__restrict__ S, const int *__restrict__ lo,
                             const int *__restrict__ hi, int h, int W, int N1, long long n,
                             const double *__restrict__ shift, double *__restrict__ out)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t / N1), j = (int)(t % N1);
        double o = -INFINITY;
        for (int w = 0; w < h; ++w) {
            if (k < lo[w] || k > hi[w]) continue;
            double v = S[((size_t)w * W + (k - lo[w])) * N1 + j];
            if (!(v > -INFINITY)) continue;
            v = __dadd_rn(v, shift[w]);
            if (o > -INFINITY) {
                const double mx = o > v ? o : v, mn = o > v ? v : o;
                o = __dsub_rn(__dadd_rn(mx, log1p(exp(__dsub_rn(mn, mx)))), EM_LN2);
            } else {
                o = v;
            }
        }
        out[t] = o;
    }
}

// normalisation: block maxima, then block sums of exp(out - max), then the shift
__global__ void k_em_max(const double *__restrict__ x, long long n, double *part)
{
    __shared__ double sh[EM_THREADS];
    double m = -INFINITY;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        m = fmax(m, x[t]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = EM_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_em_sumexp(const double *__restrict__ x, long long n, const double *part_max,
                            int nblk, double *part)
{
    __shared__ double sh[EM_THREADS];
    double mx = -INFINITY;
    for (int i = 0; i < nblk; ++i) mx = fmax(mx, part_max[i]);
    double s = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        if (x[t] > -INFINITY) s += exp(x[t] - mx);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = EM_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_em_shift(double *x, long long n, const double *part_max, const double *part_sum,
                           int nblk, double target)
{
    double mx = -INFINITY, s = 0.0;
    for (int i = 0; i < nblk; ++i) mx = fmax(mx, part_max[i]);
    for (int i = 0; i < nblk; ++i) s += part_sum[i];
    const double c = (mx + log(s)) - target;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        if (x[t] > -INFINITY) x[t] -= c;
}

int grid_for(long long n, int cap)
{
    long long b = (n + EM_THREADS - 1) / EM_THREADS;
    return (int)std::max(1LL, std::min<long long>(b, cap));
}

template <class T> T *em_alloc(size_t n, cudaError_t &e)
{
    T *p = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    return p;
}

// the join on device fragments S [h][W][N1]; lo/hi device; out device (B+1) x N1
cudaError_t join_core(const double *S, const int *d_lo, const int *d_hi, int h, int W, int B, int N1,
                      double de, double dq, double target, double *out, int *joins_host, int *ok_host,
                      cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    const int pairs = std::max(h - 1, 0);
    long long maxpts = 0;
    std::vector<int> lo(h), hi(h);
    e = cudaMemcpyAsync(lo.data(), d_lo, h * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hi.data(), d_hi, h * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    for (int p = 0; p < pairs; ++p) maxpts = std::max(maxpts, (long long)(hi[p] - lo[p + 1] + 1) * N1);
    const int nblk = grid_for(maxpts, 128);
    Best *part = em_alloc<Best>((size_t)std::max(pairs, 1) * nblk, e);
    double *shift = em_alloc<double>(h, e);
    int *joins = em_alloc<int>(2 * (size_t)std::max(pairs, 1), e);
    int *ok = em_alloc<int>(1, e);
    const long long n = (long long)(B + 1) * N1;
    const int nred = grid_for(n, 1024);
    double *pmax = em_alloc<double>(nred, e), *psum = em_alloc<double>(nred, e);
    if (e == cudaSuccess && pairs > 0) {
        k_join_cand<<<dim3(nblk, pairs), EM_THREADS, 0, st>>>(S, d_lo, d_hi, W, N1, de, dq, part);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_join_finish<<<1, 1, 0, st>>>(S, d_lo, d_hi, h, W, N1, nblk, part, shift, joins, ok);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_combine_em<<<grid_for(n, 4096), EM_THREADS, 0, st>>>(S, d_lo, d_hi, h, W, N1, n, shift, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_em_max<<<nred, EM_THREADS, 0, st>>>(out, n, pmax);
        k_em_sumexp<<<nred, EM_THREADS, 0, st>>>(out, n, pmax, nred, psum);
        k_em_shift<<<grid_for(n, 4096), EM_THREADS, 0, st>>>(out, n, pmax, psum, nred, target);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(ok_host, ok, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && joins_host && pairs > 0)
        e = cudaMemcpyAsync(joins_host, joins, 2 * (size_t)pairs * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    void *ptrs[] = {part, shift, joins, ok, pmax, psum};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    return e;
}

} // namespace

namespace rewl {
cudaError_t launch_measure_em(const State &s, cudaStream_t st)
{
    if (!s.hem) return cudaSuccess;
    const int threads = 256, blocks = (s.nw * 32 + threads - 1) / threads;
    k_measure_em<<<blocks, threads, 0, st>>>(s);
    return cudaGetLastError();
}
} // namespace rewl

extern "C" {

int rewl_get_hist_em(rewl_t r, uint32_t *out, size_t bytes)
{
    if (!r || !out) return REWL_ERR_INVALID_ARG;
    if (!r->st.hem) return r->fail(REWL_ERR_STATE, "rewl_get_hist_em: measurement is off");
    const size_t need = (size_t)r->h * r->W * (size_t)(r->N + 1) * 4u;
    if (bytes != need) return r->fail(REWL_ERR_BUFFER_TOO_SMALL, "rewl_get_hist_em: bytes != h*W*(N+1)*4");
    cudaError_t e = cudaMemcpyAsync(out, r->st.hem, need, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return r->cuda_fail(e, "rewl_get_hist_em");
    return REWL_OK;
}

int rewl_join_em(const double *S, int h, int W, int B, int N1, const int *lo_hi, double de, double dq,
                 double norm_target, double *out, int *joins, void *stream)
{
    if (!S || !out || !lo_hi || h < 1 || W < 1 || B < 1 || N1 < 2 || !(de > 0) || !(dq > 0)) {
        g_err = "rewl_join_em: invalid argument";
        return REWL_ERR_INVALID_ARG;
    }
    for (int w = 0; w < h; ++w) {
        const int lo = lo_hi[w], hi = lo_hi[h + w];
        bool bad = lo < 0 || hi > B || hi < lo || hi - lo + 1 > W;
        if (w == 0) bad |= lo != 0;
        if (w == h - 1) bad |= hi != B;
        if (w + 1 < h) bad |= lo_hi[w + 1] <= lo || lo_hi[w + 1] > hi || lo_hi[h + w + 1] < hi;
        if (bad) {
            g_err = "rewl_join_em: invalid window layout";
            return REWL_ERR_INVALID_ARG;
        }
    }
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    int *d_lohi = em_alloc<int>(2 * (size_t)h, e);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_lohi, lo_hi, 2 * (size_t)h * sizeof(int), cudaMemcpyHostToDevice, st);
    int ok = 0;
    if (e == cudaSuccess)
        e = join_core(S, d_lohi, d_lohi + h, h, W, B, N1, de, dq, norm_target, out, joins, &ok, st);
    if (d_lohi) cudaFree(d_lohi);
    if (e != cudaSuccess) {
        g_err = std::string("rewl_join_em: ") + cudaGetErrorString(e);
        return REWL_ERR_CUDA;
    }
    if (!ok) {
        g_err = "rewl_join_em: two adjacent fragments share no point";
        return REWL_ERR_NOT_CONVERGED;
    }
    return REWL_OK;
}

int rewl_stitch_em(rewl_t r, double *out, size_t n, int *joins)
{
    if (!r || !out) return REWL_ERR_INVALID_ARG;
    if (!r->st.hem) return r->fail(REWL_ERR_STATE, "rewl_stitch_em: measurement is off");
    const int N1 = r->N + 1;
    const size_t npts = (size_t)(r->B + 1) * N1;
    if (n < npts) return r->fail(REWL_ERR_BUFFER_TOO_SMALL, "rewl_stitch_em: n < (B+1)(N+1)");
    cudaError_t e = cudaSuccess;
    double *S = em_alloc<double>((size_t)r->h * r->W * N1, e);
    double *d_out = em_alloc<double>(npts, e);
    if (e == cudaSuccess) e = launch_window_mean(r->st, r->d_mean, r->stream);
    if (e == cudaSuccess) {
        k_frag_em<<<r->h * r->W, EM_THREADS, 0, r->stream>>>(r->st, r->d_mean, S);
        e = cudaGetLastError();
    }
    int ok = 0;
    if (e == cudaSuccess)
        e = join_core(S, r->st.lo, r->st.hi, r->h, r->W, r->B, N1, 4.0, 2.0,
                      (double)r->N * std::log(2.0), d_out, joins, &ok, r->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, npts * 8, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (S) cudaFree(S);
    if (d_out) cudaFree(d_out);
    if (e != cudaSuccess) return r->cuda_fail(e, "rewl_stitch_em");
    if (!ok) return r->fail(REWL_ERR_NOT_CONVERGED, "rewl_stitch_em: two adjacent fragments share no point");
    return REWL_OK;
}

} // extern "C"
