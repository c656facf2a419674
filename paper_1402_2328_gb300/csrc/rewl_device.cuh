// rewl_device.cuh -- device arithmetic of the REWL hot path (sm_103a).
//
// Philox4x32-10 counter RNG, the float64 ln u that decides moves and exchanges, the
// float32 screening value, exact sequential accumulation of ln f, and the lattice
// neighbourhood.  Every float64 operation whose rounding matters is spelled with an
// explicit __d*_rn / __fma_rn intrinsic, so no FMA contraction can change a result.
#pragma once
#include <cstdint>

namespace rewl {

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random numbers: as easy as
// 1, 2, 3").  Round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
// c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); key += Weyl constants between rounds.
// ---------------------------------------------------------------------------------------
struct u32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                         uint32_t k0, uint32_t k1)
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
        const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    return {c0, c1, c2, c3};
}

// Random-stream tags (fourth counter word = instance << 8 | tag).
enum : uint32_t { TAG_MOVE = 0u, TAG_PREP = 1u, TAG_INIT = 2u, TAG_SWAP = 3u };

__device__ __forceinline__ uint32_t mulhi(uint32_t a, uint32_t b) { return __umulhi(a, b); }

// ---------------------------------------------------------------------------------------
// ln u for u = (w + 1/2) 2^-32, float64, reproducible bit for bit:
// u = m 2^e with m in [sqrt(1/2), sqrt(2)), ln u = e ln2 + 2 atanh(s), s = (m-1)/(m+1),
// atanh(s) = s (1 + z/3 + z^2/5 + ... + z^11/23), z = s^2 <= 0.0295.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double ln64(double u)
{
    // u > 0 in the normal range (random numbers, histogram counts and their sums)
    const long long bits = __double_as_longlong(u);
    int e = (int)((bits >> 52) & 0x7ff) - 1023;
    double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    if (m > 0x1.6a09e667f3bcdp+0) {
        m = __dmul_rn(m, 0.5);
        e += 1;
    }
    const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double z = __dmul_rn(s, s);
    double p = 0x1.642c8590b2164p-5;     // 1/23
    p = __fma_rn(p, z, 0x1.8618618618618p-5); // 1/21
    p = __fma_rn(p, z, 0x1.af286bca1af28p-5); // 1/19
    p = __fma_rn(p, z, 0x1.e1e1e1e1e1e1ep-5); // 1/17
    p = __fma_rn(p, z, 0x1.1111111111111p-4); // 1/15
    p = __fma_rn(p, z, 0x1.3b13b13b13b14p-4); // 1/13
    p = __fma_rn(p, z, 0x1.745d1745d1746p-4); // 1/11
    p = __fma_rn(p, z, 0x1.c71c71c71c71cp-4); // 1/9
    p = __fma_rn(p, z, 0x1.2492492492492p-3); // 1/7
    p = __fma_rn(p, z, 0x1.999999999999ap-3); // 1/5
    p = __fma_rn(p, z, 0x1.5555555555555p-2); // 1/3
    p = __fma_rn(p, z, 1.0);
    double r = __dmul_rn(s, p);
    r = __dadd_rn(r, r);
    return __fma_rn((double)e, 0x1.62e42fefa39efp-1, r);
}

__device__ __forceinline__ double lnu64(uint32_t w)
{
    return ln64(__dmul_rn(__dadd_rn((double)w, 0.5), 0x1p-32));
}

// float32 screening value of ln u (hardware log2 approximation).  Its largest distance
// from lnu64 over all 2^32 words is measured by rewl_lnu_bound; the move kernel treats
// every decision within LNU32_EPS (plus the ln g shadow error) of the threshold with the
// float64 path, so the screen never decides a move differently.
constexpr double LNU32_EPS = 4.0e-6;

__device__ __forceinline__ float lnu32(uint32_t w)
{
    const float u = __fmaf_rn(__uint2float_rn(w), 0x1p-32f, 0x1p-33f);
    return __logf(u);
}

// x + f + f + ... (c additions, each rounded to nearest even in float64), without the loop.
// Inside one binade (x a multiple of the spacing u there) every sum x + f = x + a u + r, with
// a = floor(f/u) and 0 <= r < u, rounds to x + a u (r < u/2) or x + (a+1) u (r > u/2)
// whatever x is, so every addition that stays in the binade adds the same d and a run of them
// is one exact fma.  The addition that may leave the binade, and ties (r = u/2, whose result
// depends on the parity of x/u), are done one at a time; so are zero and tiny |x|.  For
// x < 0 the sums run towards zero and the binade ends at -2^e.
__device__ __forceinline__ double seqadd(double x, double f, uint32_t c)
{
    if (c == 0u) return x;
    if (!(f > 0.0) || !(f < INFINITY)) {
        for (uint32_t i = 0; i < c; ++i) x = __dadd_rn(x, f);
        return x;
    }
    double cf = (double)c;
    while (cf > 0.0) {
        const long long xb = __double_as_longlong(x);
        const int ex = (int)((xb >> 52) & 0x7ff);
        double n = 0.0, d = 0.0;
        if (ex > 53 && ex < 2046) {
            const double u = __longlong_as_double((long long)(ex - 52) << 52);      // ulp(x)
            const double inv_u = __longlong_as_double((long long)(2098 - ex) << 52); // 1 / u
            // the sums stay on the grid of spacing u while they lie below 2^(e+1) (x > 0) or
            // at or beyond -2^e (x < 0): D is the room left
            const double top = __longlong_as_double((long long)(x > 0.0 ? ex + 1 : ex) << 52);
            const double D = x > 0.0 ? __dsub_rn(top, x) : __dsub_rn(-x, top);
            if (f <= D) {
                const double a = floor(__dmul_rn(f, inv_u)); // f = a u + r, 0 <= r < u
                const double r = __fma_rn(-a, u, f);
                const double h = __dmul_rn(u, 0.5);
                if (r != h) { // not a tie: every addition in the binade adds d
                    d = __dmul_rn(r < h ? a : __dadd_rn(a, 1.0), u);
                    if (d == 0.0) return x; // f < u/2: no addition changes x
                    // additions j with (j+1) d + u/2 <= D stay in the binade
                    const double X = __dsub_rn(D, h);
                    if (X >= d) {
                        n = floor(__ddiv_rn(X, d));
                        if (__fma_rn(n, d, -X) > 0.0) n = __dsub_rn(n, 1.0);
                    }
                }
            }
        }
        if (n > 0.0) {
            if (cf <= n) return __fma_rn(cf, d, x); // exact: a multiple of u inside the binade
            x = __fma_rn(n, d, x);
            cf = __dsub_rn(cf, n);
        }
        x = __dadd_rn(x, f); // one addition that may leave the binade (or a tie)
        cf = __dsub_rn(cf, 1.0);
    }
    return x;
}

// Site -> (x, y) with a multiply-high by ceil(2^32 / L) (exact for site * L < 2^32).
struct Lattice {
    int L, N;
    uint32_t magic;
    __device__ __forceinline__ void nbrs(int site, int &l, int &r, int &u, int &d) const
    {
        const int y = (int)__umulhi((uint32_t)site, magic);
        const int x = site - y * L;
        const int row = site - x;
        l = (x == 0) ? site + (L - 1) : site - 1;
        r = (x == L - 1) ? row : site + 1;
        u = (y == 0) ? site + (N - L) : site - L;
        d = (y == L - 1) ? x : site + L;
    }
};

} // namespace rewl
