// rewl_kernels.cu -- the REWL hot path on sm_103a.
//
//   k_move        WL moves (Sec. 2): one warp per walker, lattice, ln g shadow and H in shared
//                 memory; 32 proposals are drawn and evaluated in parallel, then resolved in
//                 order (a proposal whose neighbourhood an earlier accepted flip touched is
//                 re-evaluated), so the result equals the one-move-at-a-time walk exactly.
//   k_check       per-walker flatness (warp-shuffle min / sum over visited bins) and window
//                 advance: average ln g over the m walkers, H = 0, ln f /= 2 (Sec. 2).
//   k_swap        replica exchange between windows (w, w+1), Eq. (1).
//   k_init_prep   seeded lattices and the walk into the window.
//   k_stitch      joining of Sec. 3, Eq. (2).
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "rewl_device.cuh"
#include "rewl_kernels.cuh"

namespace rewl {

constexpr unsigned FULL = 0xffffffffu;

__host__ __device__ inline int pad16(int n) { return (n + 15) & ~15; }
__host__ __device__ inline int padw(int w) { return (w + 3) & ~3; }

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// Energy change (in bins) of a proposal at `site` on lattice sp, plus the new state.
template <bool ISING>
__device__ __forceinline__ int propose_dk(const int8_t *sp, const Lattice &lat, int q, int site,
                                          int pr, int &snew)
{
    int l, r, u, d;
    lat.nbrs(site, l, r, u, d);
    const int s0 = sp[site];
    const int a0 = sp[l], a1 = sp[r], a2 = sp[u], a3 = sp[d];
    if (ISING) {
        snew = -s0;
        return (s0 * (a0 + a1 + a2 + a3)) / 2; // dE = 2 s0 sum, dk = dE / 4
    } else {
        int sn = s0 + 1 + pr;
        if (sn >= q) sn -= q;
        snew = sn;
        return (int)(s0 == a0) + (int)(s0 == a1) + (int)(s0 == a2) + (int)(s0 == a3) -
               (int)(sn == a0) - (int)(sn == a1) - (int)(sn == a2) - (int)(sn == a3);
    }
}

// ---------------------------------------------------------------------------------------
// WL moves.  Decision rule (Sec. 2): accept iff ln u < ln g(k) - ln g(k'), with the float64
// ln g the one-move-at-a-time walk would hold at that moment.
//
// One warp per walker.  Shared memory holds the lattice (int8), an int64 shadow
// V(b) = round(ln g0(b) 2^32) + (visits) * round(ln f 2^32) of ln g over the window, H, and one
// claim stamp per site.  Moves are taken in batches of up to 32:
//   1. lane j draws the proposal of step t+j (Philox) and evaluates its energy change on the
//      lattice as it was at the batch start; the batch is limited to its conflict-free prefix
//      (no proposal sits on the site or a neighbour of an earlier one), so those energy
//      changes stay exact whatever earlier steps of the batch do;
//   2. lane j holds, as float32 relative to the bin k0 where the batch started, ln g of bin
//      k0-16+j (+inf outside the window);
//   3. the warp walks the steps in order computing only the path: one shuffle fetches
//      ln g(k'), and the move is accepted/rejected in float32 when ln u is farther than a
//      proven error bound from ln g(k) - ln g(k'); a step inside the bound or whose k' leaves
//      the cached bins is flagged, the batch is cut there, and that one step is decided from
//      the float64 values rebuilt exactly (seqadd of the interval-start ln g and the visit
//      counts);
//   4. the side effects of the steps done (spin flips, visits of V and H) are applied
//      lane-parallel.
// At the end of the launch the float64 ln g of every bin is rebuilt exactly from its visit
// count, so the state equals that of the sequential walk bit for bit.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double shadow_error(double maxabs, int T, double lnf, bool frozen)
{
    // bound on |V(b) 2^-32 - ln g(b)| in units of 2^-32 over a launch of T moves
    const long long fb = __double_as_longlong(lnf);
    const bool dyadic = (fb & 0x000fffffffffffffLL) == 0 && lnf >= 0x1p-32;
    const double M = maxabs + (double)T * lnf;
    const int ex = (int)((__double_as_longlong(M) >> 52) & 0x7ff);
    const double ulpM = ex > 52 ? __longlong_as_double((long long)(ex - 52) << 52) : 0x1p-1022;
    if (frozen) return 0.5;
    if (dyadic) return 0.5 + 64.0 * ulpM * 0x1p32; // exact additions except binade crossings
    return 0.5 + 0.5 * (double)T + (double)T * ulpM * 0x1p31; // every addition may round
}

__device__ __forceinline__ float ulpf(float x)
{
    // unit in the last place of |x| (x normal), as a power of two
    const int e = (__float_as_int(fabsf(x)) >> 23) & 0xff;
    return e > 23 ? __int_as_float((e - 23) << 23) : 0x1p-126f;
}

__device__ __forceinline__ float warp_maxf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// visits of bin b since the launch started: the shadow grew by lnfq per visit
__device__ __forceinline__ uint32_t visits(const long long *V, const double *glng, int b, long long lnfq)
{
    return (uint32_t)((V[b] - __double2ll_rn(__dmul_rn(glng[b], 0x1p32))) / lnfq);
}

// Float64 decision from the exact values (rare): ln g of bins k and k' rebuilt by seqadd from
// the launch-start values and the visits recorded in the shadow.
__device__ __noinline__ bool exact_value_decision(const double *glng, const long long *V, int lo,
                                                  int k, int kp, double lnf, long long lnfq,
                                                  bool frozen, uint32_t w2)
{
    const uint32_t vk = frozen ? 0u : visits(V, glng, k - lo, lnfq);
    const uint32_t vkp = frozen ? 0u : visits(V, glng, kp - lo, lnfq);
    const double lk = seqadd(glng[k - lo], lnf, vk);
    const double lkp = seqadd(glng[kp - lo], lnf, vkp);
    const double d = __dsub_rn(lk, lkp);
    return (d >= 0.0) || (lnu64(w2) < d);
}

// The same, for the warp of one walker: every lane takes part after the lanes' shadow updates.
__device__ __forceinline__ bool exact_decision(const double *glng, const long long *V, int lo, int k,
                                               int kp, double lnf, long long lnfq, bool frozen,
                                               uint32_t w2)
{
    __syncwarp();
    return exact_value_decision(glng, V, lo, k, kp, lnf, lnfq, frozen, w2);
}

// One walker's `c.T` moves; `base` is the walker's shared-memory block, the whole warp calls.
template <bool ISING, bool REPLAY, bool CHECK>
__device__ __forceinline__ void move_walker(const State &s, const MoveCfg &c, const int slot,
                                            unsigned char *base, const int lane)
{
    if (s.status != nullptr && s.status->done) return;
    int8_t *sp = reinterpret_cast<int8_t *>(base);
    long long *V = reinterpret_cast<long long *>(base + pad16(s.N));
    uint32_t *vis = reinterpret_cast<uint32_t *>(V + padw(s.W));      // [W bits] bin visited
    uint16_t *stamp = reinterpret_cast<uint16_t *>(vis + visw(s.W));  // [N] batch claims

    const int w = slot / s.m;
    const int lo = s.lo[w], hi = s.hi[w], nb = hi - lo + 1;
    int k = s.k[slot];
    if (lo < 0 || nb < 1 || nb > s.W || k < lo || k > hi) { // malformed input: refuse
        if (lane == 0) atomicOr(&s.status->err, ERR_INPUT);
        return;
    }
    const double lnf = s.lnf[w];
    const bool frozen = s.finished[w] != 0;
    const int cfg = s.cfg ? s.cfg[slot] : slot;
    int8_t *gsp = s.spins + (size_t)cfg * s.spin_stride;
    const double *glng = s.lng + (size_t)slot * s.W;
    uint32_t *gH = s.H + (size_t)slot * s.W;
    const Lattice lat{s.L, s.N, s.magic};
    const int T = c.T;

    // ---- load lattice, shadow ln g, H; clear the claim stamps
    if (s.vec_spins) {
        const int4 *src = reinterpret_cast<const int4 *>(gsp);
        int4 *dst = reinterpret_cast<int4 *>(sp);
        for (int i = lane; i < (s.N >> 4); i += 32) dst[i] = src[i];
    } else {
        for (int i = lane; i < s.N; i += 32) sp[i] = gsp[i];
    }
    for (int i = lane; i < s.N; i += 32) stamp[i] = 0xffffu; // matches no batch
    double mx = 0.0;
    bool bad = false;
    for (int b = lane; b < nb; b += 32) {
        const double x = glng[b];
        bad = bad || !(fabs(x) < 0x1p30); // also catches NaN
        mx = fmax(mx, fabs(x));
        V[b] = bad ? 0LL : __double2ll_rn(__dmul_rn(x, 0x1p32));
    }
    // visited bits: the bins any walker of the window had visited when this launch started,
    // the start bin, and every bin this walker enters for the first time (always through the
    // float64 path below)
    // (replay has no window mask: every bin counts as visited there)
    const uint8_t *gmask = s.mask ? s.mask + (size_t)w * s.W : nullptr;
    for (int i = 0; i < visw(s.W); ++i) { // word i: bins 32i .. 32i+31, one per lane
        const int b = 32 * i + lane;
        const unsigned bits = __ballot_sync(FULL, b < nb && (gmask == nullptr || gmask[b]));
        if (lane == 0) vis[i] = bits;
    }
    __syncwarp();
    if (lane == 0) vis[(k - lo) >> 5] |= 1u << ((k - lo) & 31); // the start bin
    mx = warp_max(mx);
    // the shadow of a running window ends the launch below (max |ln g| + T ln f) 2^32 < 2^62,
    // and ln f 2^32 must not round to zero; a frozen window adds nothing to it
    const bool lnf_ok = frozen || (lnf >= 0x1p-32 && lnf < 0x1p20 && mx + (double)T * lnf < 0x1p30);
    if (__any_sync(FULL, bad) || !lnf_ok) {
        // the int64 shadow would overflow or lose the increment: leave the state untouched
        if (lane == 0) atomicOr(&s.status->err, ERR_RANGE);
        return;
    }
    const long long lnfq = __double2ll_rn(__dmul_rn(lnf, 0x1p32));
    // interval-constant part of the float32 screening margin (ln units)
    const float Mbase = (float)(c.eps_l + 2.0 * shadow_error(mx, T, lnf, frozen) * 0x1p-32) + 0x1p-21f;
    const float lnf_f = frozen ? 0.0f : (float)lnf;
    __syncwarp();

    const unsigned long long st0 = s.step[slot];
    unsigned int nacc = 0, nex = 0, nmis = 0;
    const uint32_t tag = (s.inst << 8) | TAG_MOVE;

    int t = 0;
    unsigned batch = 0;
    while (t < T) {
        ++batch;
        const int n = min(32, T - t);
        // ---- register cache of ln g around k0 (float32, relative to bin k0)
        const int k0 = k, base = k0 - 16;
        const int bj = base + lane;
        const bool bin_ok = bj >= lo && bj <= hi;
        float Lw = 0.0f;
        if (bin_ok) {
            const long long x = V[bj - lo] - V[k0 - lo];
            Lw = __fmaf_rn(__uint2float_rn((uint32_t)x), 0x1p-32f, (float)(int)(x >> 32));
        }
        // largest |Lw| of the cache (non-negative floats order like their bit patterns)
        // Bins never visited keep their initial ln g while the others grow, so their cache
        // values can be far off: they are marked NaN (a step there is flagged unsure and
        // decided from the float64 values) and do not widen every other step's margin.
        const bool far = bin_ok && !((vis[(bj - lo) >> 5] >> ((bj - lo) & 31)) & 1u);
        const float Mx = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(bin_ok && !far ? fabsf(Lw) : 0.0f))) +
                         33.0f * lnf_f + 0x1p-20f;
        const float M = Mbase + 40.0f * ulpf(2.0f * Mx);
        if (!bin_ok) Lw = INFINITY; // a move there is rejected: ln g(k) - inf < ln u
        if (far) Lw = __int_as_float(0x7fc00000);

        // ---- parallel phase: lane j evaluates proposal t + j on the batch-start lattice
        uint32_t w0, w1, w2;
        if (REPLAY) {
            if (lane < n) {
                const uint32_t *wp = c.words + ((size_t)slot * T + t + lane) * 3;
                w0 = wp[0];
                w1 = wp[1];
                w2 = wp[2];
            } else {
                w0 = w1 = w2 = 0u;
            }
        } else {
            const unsigned long long sn = st0 + (unsigned long long)(t + lane);
            const u32x4 r = philox((uint32_t)sn, (uint32_t)(sn >> 32), (uint32_t)(s.slot0 + slot),
                                   tag, s.key0, s.key1);
            w0 = r.x;
            w1 = r.y;
            w2 = r.z;
        }
        const int site = (int)mulhi(w0, (uint32_t)s.N);
        int nl, nr, nu, nd;
        lat.nbrs(site, nl, nr, nu, nd);
        const int pr = ISING ? 0 : (int)mulhi(w1, (uint32_t)(s.q - 1));
        int snew;
        const int dk = propose_dk<ISING>(sp, lat, s.q, site, pr, snew);
        // a proposal that keeps the energy is always accepted and keeps the bin: the serial
        // walk sees it as a sure non-move (threshold +inf), the lane itself records the flip
        const bool dz = dk == 0;
        const float thr = dz ? INFINITY : lnu32(w2);
        // conflict-free prefix: proposal j may be resolved on the batch-start lattice only if
        // no earlier proposal of the batch sits on its site or a neighbour.
        // Claim stamp = (batch mod 2047) << 5 | lane of the lowest lane proposing the site: every
        // lane writes its stamp, then a lane that finds a later lane's stamp on its site writes
        // again until none does (at most one extra pass unless three lanes share a site).  A
        // stale stamp of an old batch with the same low bits can only cut a batch early.
        const unsigned btag = batch % 2047u;
        const uint16_t mystamp = (uint16_t)((btag << 5) | (unsigned)lane);
        if (lane < n) stamp[site] = mystamp;
        __syncwarp();
        for (int it = 0; it < 32; ++it) { // each pass lowers some stamp: ends within 32 passes
            bool again = false;
            if (lane < n) {
                const unsigned v = stamp[site];
                again = (v >> 5) == btag && (int)(v & 31u) > lane;
            }
            __syncwarp();
            if (!__any_sync(FULL, again)) break;
            if (again) stamp[site] = mystamp;
            __syncwarp();
        }
        bool conflict = false;
        {
            const int xs[5] = {site, nl, nr, nu, nd};
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                const unsigned v = stamp[xs[m]];
                conflict = conflict || ((v >> 5) == btag && (int)(v & 31u) < lane);
            }
        }
        const unsigned cmask = __ballot_sync(FULL, conflict && lane < n);
        const int J = cmask ? (__ffs(cmask) - 1) : n; // >= 1: lane 0 never conflicts

        // ---- serial phase: the path k_0, k_1, ... only.  Every step runs unconditionally;
        // lane j records the bin after step j and whether step j was too close to call in
        // float32, and the batch is cut at the first such step afterwards (the steps after it
        // are discarded), so no bookkeeping sits on the dependency chain.
        // Steps are resolved in pairs (2p, 2p+1): the three cache lookups a pair can need
        // (k' of the first step; k' of the second step after the first moved / stayed) are
        // issued together and the second step is evaluated in both worlds, so one shuffle
        // latency and one select cover two moves.  Decision variable:
        // e = ln g(k) - ln g(k') - thr; accept if e > M, reject if e < -M, else unsure.
        // A target outside the 32 cached bins reads a wrong lane; such steps are found after
        // the loop (the target is known per lane) and cut there as well.
        int myx = 16;      // lane j: cache offset of the bin after step j
        bool myun = false; // lane j: step j unsure in float32
        bool mysa = false, mysr = false; // CHECK: float32 verdict of step j (sure accept / reject)
        int xk = 16;       // cache offset of the current bin
        float Lk = 0.0f;   // running value of the current bin (the cache holds it only once left)
#pragma unroll
        for (int p = 0; p < 16; ++p) {
            const int i = 2 * p;
            if ((p & 1) == 0 && p > 0 && (i >= J || (unsigned)xk >= 32u || __any_sync(FULL, myun)))
                break; // every 2 pairs
            const int dk0 = __shfl_sync(FULL, dk, i), dk1 = __shfl_sync(FULL, dk, i + 1);
            const float th0 = __shfl_sync(FULL, thr, i), th1 = __shfl_sync(FULL, thr, i + 1);
            const int x0 = xk + dk0; // k' of step i
            const int xA = x0 + dk1; // k' of step i+1 if step i moved
            const int xR = xk + dk1; // k' of step i+1 if step i stayed
            const bool atk = lane == xk, at0 = lane == x0;
            const float L0 = __shfl_sync(FULL, Lw, x0 & 31);
            const float LA_ = __shfl_sync(FULL, Lw, xA & 31);
            const float LR = __shfl_sync(FULL, Lw, xR & 31);
            const float LA = (dk1 == -dk0) ? Lk : LA_; // back to the bin just left
            const float Lm = L0 + lnf_f;               // value after step i if moved
            const float Ls = Lk + lnf_f;               // value after step i if stayed
            // step i
            const float e0 = (Lk - L0) - th0;
            const bool m0 = e0 > M;
            const bool un0 = CHECK ? (th0 != INFINITY && L0 != INFINITY) : !(fabsf(e0) > M);
            // step i+1 in both worlds, then the world step i chose
            const float e1A = (Lm - LA) - th1;
            const float e1R = (Ls - LR) - th1;
            const bool m1 = m0 ? (e1A > M) : (e1R > M);
            const float e1 = m0 ? e1A : e1R;
            const float L1 = m0 ? LA : LR;
            const float Lc1 = m0 ? Lm : Ls;
            const int x1 = m0 ? xA : xR;
            const int xc1 = m0 ? x0 : xk;
            const bool un1 = CHECK ? (th1 != INFINITY && L1 != INFINITY) : !(fabsf(e1) > M);
            // the bins left keep their running values
            if (m0 && atk) Lw = Lk;
            if (m1 && (m0 ? at0 : atk)) Lw = Lc1;
            if (lane == i) {
                myx = xc1;
                myun = un0;
                if (CHECK) {
                    mysa = e0 > M;
                    mysr = e0 < -M;
                }
            }
            xk = m1 ? x1 : xc1;
            if (lane == i + 1) {
                myx = xk;
                myun = un1;
                if (CHECK) {
                    mysa = e1 > M;
                    mysr = e1 < -M;
                }
            }
            Lk = (m1 ? L1 : Lc1) + lnf_f;
        }
        // bin before step j; a target outside the cache makes step j unsure as well
        const int xup = __shfl_up_sync(FULL, myx, 1);
        const int xbefore = lane == 0 ? 16 : xup;
        const bool oob = (unsigned)(xbefore + dk) >= 32u;
        const unsigned badbits = __ballot_sync(FULL, myun || oob);
        const unsigned stopbits = badbits | (J >= 32 ? 0u : (0xffffffffu << J));
        const int ndone = stopbits ? __ffs(stopbits) - 1 : 32;
        const bool amb_stop = ndone < J;
        if (ndone == 0 && !amb_stop) { // no step done and none to decide: cannot happen (J >= 1)
            if (lane == 0) atomicOr(&s.status->err, ERR_INPUT);
            return;
        }
        // bin after each step (valid for the steps done, all inside the cache)
        const int mypos = k0 - 16 + myx;
        const int kc = ndone > 0 ? k0 - 16 + __shfl_sync(FULL, myx, ndone - 1) : k0;
        // float32 verdict at the cut (CHECK): 1 sure accept, 0 sure reject, -1 unsure
        int scr = -1;
        if (CHECK) {
            const unsigned sa = __ballot_sync(FULL, mysa), sr = __ballot_sync(FULL, mysr);
            scr = ndone >= 32 ? -1 : (((sa >> ndone) & 1u) ? 1 : (((sr >> ndone) & 1u) ? 0 : -1));
        }

        // ---- side effects of steps 0..ndone-1
        const bool mine = lane < ndone;
        const bool accj = dz || myx != xbefore; // step j accepted (a move to another bin, or dE = 0)
        if (mine && accj) sp[site] = (int8_t)snew; // conflict-free sites
        {
            // visits: the lanes of one bin add their count with one plain update (no atomics)
            const unsigned grp = __match_any_sync(FULL, mine ? mypos : -1 - lane);
            if (mine && !frozen && lane == __ffs(grp) - 1)
                V[mypos - lo] += (long long)__popc(grp) * lnfq;
        }
        if (REPLAY && mine) {
            c.acc_out[(size_t)slot * T + t + lane] = accj ? 1 : 0;
            c.dk_out[(size_t)slot * T + t + lane] = dk;
        }
        nacc += __popc(__ballot_sync(FULL, mine && accj));
        k = kc;
        t += ndone;
        __syncwarp();

        // ---- a proposal too close to call in float32: decide it from the float64 values
        if (amb_stop) {
            const int i = ndone;
            const int dki = __shfl_sync(FULL, dk, i);
            const int sitei = __shfl_sync(FULL, site, i);
            const int snewi = __shfl_sync(FULL, snew, i);
            const uint32_t w2i = __shfl_sync(FULL, w2, i);
            const int kp = k + dki;
            bool acc = dki == 0;
            if (!acc && kp >= lo && kp <= hi) {
                acc = exact_decision(glng, V, lo, k, kp, lnf, lnfq, frozen, w2i);
                if (scr < 0) ++nex;
                else if ((int)acc != scr) ++nmis;
            }
            if (acc) {
                sp[sitei] = (int8_t)snewi;
                k = kp;
                ++nacc;
            }
            if (!frozen && lane == 0) V[k - lo] += lnfq;
            // a bin reached for the first time is only ever entered here (its cache value is
            // NaN until marked), so marking it here keeps the visited set complete
            if (lane == 0) vis[(k - lo) >> 5] |= 1u << ((k - lo) & 31);
            if (REPLAY && lane == 0) {
                c.acc_out[(size_t)slot * T + t] = acc ? 1 : 0;
                c.dk_out[(size_t)slot * T + t] = dki;
            }
            t += 1;
            __syncwarp();
        }
    }

    // ---- write back lattice, float64 ln g (rebuilt exactly), H, counters
    if (s.vec_spins) {
        const int4 *src = reinterpret_cast<const int4 *>(sp);
        int4 *dst = reinterpret_cast<int4 *>(gsp);
        for (int i = lane; i < (s.N >> 4); i += 32) dst[i] = src[i];
    } else {
        for (int i = lane; i < s.N; i += 32) gsp[i] = sp[i];
    }
    if (!frozen) {
        double *gl = s.lng + (size_t)slot * s.W;
        for (int b = lane; b < nb; b += 32) {
            const uint32_t v = visits(V, gl, b, lnfq);
            if (v != 0u) {
                gl[b] = seqadd(gl[b], lnf, v);
                gH[b] += v;
            }
        }
    }
    if (lane == 0) {
        s.k[slot] = k;
        s.step[slot] = st0 + (unsigned long long)T;
        s.acc[slot] += nacc;
        if (nex) atomicAdd(&s.status->n_exact, (unsigned long long)nex);
        if (nmis) atomicAdd(&s.status->n_mismatch, (unsigned long long)nmis);
    }
}

// ---------------------------------------------------------------------------------------
// One thread per walker (small lattices, many walkers): the plain sequential walk of Sec. 2.
// ln g is the same int64 shadow as above (multiples of 2^-32, exact visit counts), held in
// shared memory; the current bin's value stays in registers.  Each decision is screened in
// fixed point: D = V(k) - V(k') against ln u 2^32 (the float32 value, converted exactly up to
// one unit), accepted or rejected when |D - ln u 2^32| exceeds the margin Mq that bounds the
// shadow error, the float32 ln u error and the float64 rounding of ln g(k) - ln g(k'); inside
// the margin the float64 values are rebuilt (rare).  No float arithmetic in the loop, no
// warp cooperation: the 32 walkers of a warp run in lockstep, each on its own data.
// ---------------------------------------------------------------------------------------
template <bool ISING, bool REPLAY, bool CHECK>
__device__ __forceinline__ void move_walker_thread(const State &s, const MoveCfg &c, const int slot,
                                                   unsigned char *base)
{
    if (s.status != nullptr && s.status->done) return;
    int8_t *sp = reinterpret_cast<int8_t *>(base);
    long long *V = reinterpret_cast<long long *>(base + pad16(s.N));
    const int w = slot / s.m;
    const int lo = s.lo[w], hi = s.hi[w], nb = hi - lo + 1;
    int k = s.k[slot];
    if (lo < 0 || nb < 1 || nb > s.W || k < lo || k > hi) {
        atomicOr(&s.status->err, ERR_INPUT);
        return;
    }
    const double lnf = s.lnf[w];
    const bool frozen = s.finished[w] != 0;
    const int cfg = s.cfg ? s.cfg[slot] : slot;
    int8_t *gsp = s.spins + (size_t)cfg * s.spin_stride;
    double *glng = s.lng + (size_t)slot * s.W;
    uint32_t *gH = s.H + (size_t)slot * s.W;
    const Lattice lat{s.L, s.N, s.magic};
    const int T = c.T;
    if (s.vec_spins) {
        const int4 *src = reinterpret_cast<const int4 *>(gsp);
        int4 *dst = reinterpret_cast<int4 *>(sp);
        for (int i = 0; i < (s.N >> 4); ++i) dst[i] = src[i];
    } else {
        for (int i = 0; i < s.N; ++i) sp[i] = gsp[i];
    }
    double mx = 0.0;
    bool bad = false;
    for (int b = 0; b < nb; ++b) {
        const double x = glng[b];
        bad = bad || !(fabs(x) < 0x1p30);
        mx = fmax(mx, fabs(x));
        V[b] = bad ? 0LL : __double2ll_rn(__dmul_rn(x, 0x1p32));
    }
    const bool lnf_ok = frozen || (lnf >= 0x1p-32 && lnf < 0x1p20 && mx + (double)T * lnf < 0x1p30);
    if (bad || !lnf_ok) {
        atomicOr(&s.status->err, ERR_RANGE);
        return;
    }
    const long long lnfq = frozen ? 0LL : __double2ll_rn(__dmul_rn(lnf, 0x1p32));
    // margin in units of 2^-32: both shadow values, the float32 ln u, the float64 difference
    // of ln g values below 2^31 (half an ulp, 2^-22) and the conversion of ln u (one unit)
    const long long Mq = (long long)(2.0 * shadow_error(mx, T, lnf, frozen) + (c.eps_l + 0x1p-21) * 0x1p32) + 4;
    const unsigned long long st0 = s.step[slot];
    const uint32_t tag = (s.inst << 8) | TAG_MOVE;
    unsigned int nacc = 0, nex = 0, nmis = 0;
    long long Vk = V[k - lo];
    for (int t = 0; t < T; ++t) {
        uint32_t w0, w1, w2;
        if (REPLAY) {
            const uint32_t *wp = c.words + ((size_t)slot * T + t) * 3;
            w0 = wp[0];
            w1 = wp[1];
            w2 = wp[2];
        } else {
            const unsigned long long sn = st0 + (unsigned long long)t;
            const u32x4 r = philox((uint32_t)sn, (uint32_t)(sn >> 32), (uint32_t)(s.slot0 + slot),
                                   tag, s.key0, s.key1);
            w0 = r.x;
            w1 = r.y;
            w2 = r.z;
        }
        const int site = (int)mulhi(w0, (uint32_t)s.N);
        const int pr = ISING ? 0 : (int)mulhi(w1, (uint32_t)(s.q - 1));
        int snew;
        const int dk = propose_dk<ISING>(sp, lat, s.q, site, pr, snew);
        const int kp = k + dk;
        bool acc = dk == 0;
        if (!acc && kp >= lo && kp <= hi) {
            const long long e = (Vk - V[kp - lo]) - (long long)__float2ll_rz(lnu32(w2) * 0x1p32f);
            const int scr = e > Mq ? 1 : (e < -Mq ? 0 : -1);
            if (scr >= 0 && !CHECK) {
                acc = scr == 1;
            } else {
                V[k - lo] = Vk;
                acc = exact_value_decision(glng, V, lo, k, kp, lnf, lnfq, frozen, w2);
                if (scr < 0) ++nex;
                else if ((int)acc != scr) ++nmis;
            }
        }
        if (acc) {
            sp[site] = (int8_t)snew;
            if (dk != 0) {
                V[k - lo] = Vk;
                k = kp;
                Vk = V[k - lo];
            }
            ++nacc;
        }
        Vk += lnfq; // ln g(k) += ln f, H(k)++: one visit of the current bin
        if (REPLAY) {
            c.acc_out[(size_t)slot * T + t] = acc ? 1 : 0;
            c.dk_out[(size_t)slot * T + t] = dk;
        }
    }
    V[k - lo] = Vk;
    if (s.vec_spins) {
        const int4 *src = reinterpret_cast<const int4 *>(sp);
        int4 *dst = reinterpret_cast<int4 *>(gsp);
        for (int i = 0; i < (s.N >> 4); ++i) dst[i] = src[i];
    } else {
        for (int i = 0; i < s.N; ++i) gsp[i] = sp[i];
    }
    if (!frozen)
        for (int b = 0; b < nb; ++b) {
            const uint32_t v = visits(V, glng, b, lnfq);
            if (v != 0u) {
                glng[b] = seqadd(glng[b], lnf, v);
                gH[b] += v;
            }
        }
    s.k[slot] = k;
    s.step[slot] = st0 + (unsigned long long)T;
    s.acc[slot] += nacc;
    if (nex) atomicAdd(&s.status->n_exact, (unsigned long long)nex);
    if (nmis) atomicAdd(&s.status->n_mismatch, (unsigned long long)nmis);
}

template <bool ISING, bool REPLAY, bool CHECK>
__global__ void __launch_bounds__(256) k_move_thread(State s, MoveCfg c)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int slot = blockIdx.x * c.walkers_per_block + threadIdx.x;
    if (threadIdx.x >= c.walkers_per_block || slot >= s.nw) return;
    move_walker_thread<ISING, REPLAY, CHECK>(s, c, slot,
                                             smem + (size_t)threadIdx.x * move_smem_per_thread_walker(s.N, s.W));
}

template <bool ISING, bool REPLAY, bool CHECK>
__global__ void __launch_bounds__(512, 1) k_move(State s, MoveCfg c)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int slot = blockIdx.x * c.walkers_per_block + wib;
    if (slot >= s.nw) return;
    move_walker<ISING, REPLAY, CHECK>(s, c, slot, smem + (size_t)wib * move_smem_per_walker(s.N, s.W),
                                      lane);
}

// Batched instances in one launch: CTA b serves walkers jobs[b].y .. jobs[b].y + jobs[b].z - 1 of
// instance jobs[b].x & 0xffffff, one warp per walker, or one thread per walker when bit 24 of
// jobs[b].x is set; the model and the layout are chosen per CTA.
template <bool CHECK>
__global__ void __launch_bounds__(512, 1) k_move_batch(const State *__restrict__ states,
                                                    const int4 *__restrict__ jobs, MoveCfg c)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int4 job = jobs[blockIdx.x];
    const State s = states[job.x & 0xffffff];
    if (job.x >> 24) { // one thread per walker
        const int t = threadIdx.x;
        if (t >= job.z) return;
        unsigned char *base = smem + (size_t)t * move_smem_per_thread_walker(s.N, s.W);
        if (s.model == 0) move_walker_thread<true, false, CHECK>(s, c, job.y + t, base);
        else move_walker_thread<false, false, CHECK>(s, c, job.y + t, base);
        return;
    }
    if (wib >= job.z) return;
    unsigned char *base = smem + (size_t)wib * move_smem_per_walker(s.N, s.W);
    if (s.model == 0) move_walker<true, false, CHECK>(s, c, job.y + wib, base, lane);
    else move_walker<false, false, CHECK>(s, c, job.y + wib, base, lane);
}

cudaError_t launch_move_batch(const State *states, const int4 *jobs, int njobs, int walkers_per_block,
                              size_t smem, const MoveCfg &c, cudaStream_t st)
{
    if (njobs <= 0) return cudaSuccess;
    cudaError_t e;
    if (c.check_all) {
        e = cudaFuncSetAttribute(k_move_batch<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_move_batch<true><<<njobs, 32 * walkers_per_block, smem, st>>>(states, jobs, c);
    } else {
        e = cudaFuncSetAttribute(k_move_batch<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_move_batch<false><<<njobs, 32 * walkers_per_block, smem, st>>>(states, jobs, c);
    }
    return cudaGetLastError();
}

cudaError_t launch_move(const State &s, const MoveCfg &c, cudaStream_t st)
{
    if (c.layout == 1) { // one thread per walker, c.walkers_per_block walkers (threads) per CTA
        const int G = c.walkers_per_block;
        const size_t smem = (size_t)G * move_smem_per_thread_walker(s.N, s.W);
        const dim3 grid((s.nw + G - 1) / G), block((G + 31) & ~31);
        const bool ising = s.model == 0;
        cudaError_t e;
#define REWL_LAUNCH_MOVE_T(I, R, C)                                                              \
    do {                                                                                         \
        e = cudaFuncSetAttribute(k_move_thread<I, R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)smem);                                                     \
        if (e != cudaSuccess) return e;                                                          \
        k_move_thread<I, R, C><<<grid, block, smem, st>>>(s, c);                                 \
    } while (0)
        if (ising) {
            if (c.words) REWL_LAUNCH_MOVE_T(true, true, false);
            else if (c.check_all) REWL_LAUNCH_MOVE_T(true, false, true);
            else REWL_LAUNCH_MOVE_T(true, false, false);
        } else {
            if (c.words) REWL_LAUNCH_MOVE_T(false, true, false);
            else if (c.check_all) REWL_LAUNCH_MOVE_T(false, false, true);
            else REWL_LAUNCH_MOVE_T(false, false, false);
        }
#undef REWL_LAUNCH_MOVE_T
        return cudaGetLastError();
    }
    const int G = c.walkers_per_block;
    const size_t smem = (size_t)G * move_smem_per_walker(s.N, s.W);
    const dim3 grid((s.nw + G - 1) / G), block(32 * G);
    const bool ising = s.model == 0;
    cudaError_t e;
#define REWL_LAUNCH_MOVE(I, R, C)                                                                \
    do {                                                                                         \
        e = cudaFuncSetAttribute(k_move<I, R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                 (int)smem);                                                     \
        if (e != cudaSuccess) return e;                                                          \
        k_move<I, R, C><<<grid, block, smem, st>>>(s, c);                                        \
    } while (0)
    if (ising) {
        if (c.words) REWL_LAUNCH_MOVE(true, true, false);
        else if (c.check_all) REWL_LAUNCH_MOVE(true, false, true);
        else REWL_LAUNCH_MOVE(true, false, false);
    } else {
        if (c.words) REWL_LAUNCH_MOVE(false, true, false);
        else if (c.check_all) REWL_LAUNCH_MOVE(false, false, true);
        else REWL_LAUNCH_MOVE(false, false, false);
    }
#undef REWL_LAUNCH_MOVE
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Seeded lattices and prep into the window (one thread per walker; runs once).
// ---------------------------------------------------------------------------------------
__device__ int bin_of_lattice(const int8_t *sp, int L, int N, bool ising)
{
    long long E = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            const int a = sp[y * L + x];
            const int r = sp[y * L + (x + 1 == L ? 0 : x + 1)];
            const int d = sp[(y + 1 == L ? 0 : y + 1) * L + x];
            if (ising) E -= (long long)(a * r + a * d);
            else E -= (long long)((a == r) + (a == d));
        }
    return ising ? (int)((E + 2LL * N) / 4) : (int)(E + 2LL * N);
}

__device__ __forceinline__ int dist_to(int k, int lo, int hi)
{
    return k < lo ? lo - k : (k > hi ? k - hi : 0);
}

__global__ void k_init_prep(State s, long long prep_budget)
{
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= s.nw) return;
    const bool ising = s.model == 0;
    const int w = slot / s.m, lo = s.lo[w], hi = s.hi[w], N = s.N;
    int8_t *sp = s.spins + (size_t)slot * s.spin_stride; // cfg[slot] == slot at start
    const Lattice lat{s.L, N, s.magic};
    for (int c = 0; 4 * c < N; ++c) {
        const u32x4 r = philox((uint32_t)c, 0u, (uint32_t)(s.slot0 + slot), (s.inst << 8) | TAG_INIT,
                               s.key0, s.key1);
        const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
        for (int j = 0; j < 4 && 4 * c + j < N; ++j)
            sp[4 * c + j] = ising ? (int8_t)((wv[j] >> 31) ? -1 : 1)
                                  : (int8_t)mulhi(wv[j], (uint32_t)s.q);
    }
    int k = bin_of_lattice(sp, s.L, N, ising);
    unsigned long long ps = 0;
    const unsigned long long budget = (unsigned long long)prep_budget * (unsigned long long)N;
    int restarts = 0;
    for (int phase = 0; phase < 2 && dist_to(k, lo, hi) > 0; ++phase) {
        if (phase == 1) { // restart from the ground state, or the checkerboard for an upper window
            const bool top = 2 * lo > (ising ? N : 2 * N);
            for (int j = 0; j < N; ++j) {
                const bool odd = top && (((j % s.L) + (j / s.L)) & 1);
                sp[j] = ising ? (int8_t)(odd ? -1 : 1) : (int8_t)(odd ? 1 : 0);
            }
            k = top ? bin_of_lattice(sp, s.L, N, ising) : 0;
            ++restarts;
        }
        const unsigned long long end = ps + budget;
        while (dist_to(k, lo, hi) > 0 && ps < end) {
            const u32x4 r = philox((uint32_t)ps, (uint32_t)(ps >> 32), (uint32_t)(s.slot0 + slot),
                                   (s.inst << 8) | TAG_PREP, s.key0, s.key1);
            const int site = (int)mulhi(r.x, (uint32_t)N);
            int snew, dk;
            if (ising) dk = propose_dk<true>(sp, lat, s.q, site, 0, snew);
            else dk = propose_dk<false>(sp, lat, s.q, site, (int)mulhi(r.y, (uint32_t)(s.q - 1)), snew);
            if (dist_to(k + dk, lo, hi) <= dist_to(k, lo, hi)) {
                sp[site] = (int8_t)snew;
                k += dk;
            }
            ++ps;
        }
    }
    s.k[slot] = k;
    s.cfg[slot] = slot;
    s.pstep[slot] = ps;
    s.restarts[slot] = restarts;
    if (dist_to(k, lo, hi) > 0) atomicOr(&s.status->err, ERR_PREP);
}

cudaError_t launch_init_prep(const State &s, long long prep_budget, cudaStream_t st)
{
    k_init_prep<<<(s.nw + 63) / 64, 64, 0, st>>>(s, prep_budget);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Flatness + window advance (Sec. 2).  One CTA per window.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void check_window(const State &s, const int w, const double flatness,
                                             const double lnf_final)
{
    if (s.status->done || s.finished[w]) return;
    const int m = s.m, W = s.W, nb = s.hi[w] - s.lo[w] + 1;
    uint8_t *mask = s.mask + (size_t)w * W;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        if (mask[b]) continue;
        uint32_t any = 0u; // the m loads are independent, so they overlap
#pragma unroll 8
        for (int i = 0; i < m; ++i) any |= s.H[(size_t)(w * m + i) * W + b];
        if (any) mask[b] = 1;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // visited bins of the window (for t of the 1/t schedule)
    __shared__ int nvis_w[32];
    int nv = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) nv += mask[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nv += __shfl_xor_sync(FULL, nv, o);
    if (lane == 0) nvis_w[wid] = nv;
    const bool tmode = s.mode[w] != 0;
    __shared__ int notflat; // walkers of the window not (yet) flat
    if (threadIdx.x == 0) notflat = 0;
    __syncthreads();
    for (int i = wid; i < m && !tmode; i += nwarp) {
        const int g = w * m + i;
        if (s.flat[g]) continue;
        const uint32_t *H = s.H + (size_t)g * W;
        unsigned long long sum = 0;
        uint32_t mn = 0xffffffffu;
        int cnt = 0;
#pragma unroll 4
        for (int b = lane; b < nb; b += 32) { // both loads unconditional: they overlap
            const uint32_t v = H[b];
            if (mask[b]) {
                sum += v;
                mn = min(mn, v);
                ++cnt;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(FULL, sum, o);
            mn = min(mn, __shfl_xor_sync(FULL, mn, o));
            cnt += __shfl_xor_sync(FULL, cnt, o);
        }
        if (lane == 0) {
            if (cnt > 0 && __dmul_rn((double)mn, (double)cnt) >= __dmul_rn(flatness, (double)sum))
                s.flat[g] = 1;
            else
                atomicAdd(&notflat, 1);
        }
    }
    __syncthreads();
    if (notflat != 0) return; // 1/t mode: every check averages and sets ln f = 1/t
    // ln f after this advance (every thread computes the same value)
    long long nvis = 0;
    for (int i = 0; i < nwarp; ++i) nvis += nvis_w[i];
    // 1/t with t = moves per walker / visited bins, i.e. ln f = visited bins / moves
    const double inv_t = nvis > 0 ? __ddiv_rn((double)nvis, (double)s.step[w * m]) : 0.0;
    bool to_t = false;
    double nl;
    if (tmode) {
        nl = inv_t;
    } else {
        nl = __dmul_rn(s.lnf[w], 0.5);
        if (s.schedule == 1 && nl < inv_t) {
            to_t = true;
            nl = inv_t;
        }
    }
    // a window about to finish keeps its walkers' last fragments (resampling error bars, Sec. 3)
    const bool finishing = nl < lnf_final;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < m; ++i) acc = __dadd_rn(acc, s.lng[(size_t)(w * m + i) * W + b]);
        const double avg = __ddiv_rn(acc, (double)m);
        for (int i = 0; i < m; ++i) {
            if (finishing) s.frag[(size_t)(w * m + i) * W + b] = s.lng[(size_t)(w * m + i) * W + b];
            s.lng[(size_t)(w * m + i) * W + b] = avg;
            s.H[(size_t)(w * m + i) * W + b] = 0u;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < m; ++i) s.flat[w * m + i] = 0;
        if (to_t) s.mode[w] = 1;
        s.lnf[w] = nl;
        if (s.iter[w] == 0) s.it1_round[w] = s.status->round + 1;
        s.iter[w] += 1;
        if (finishing) s.finished[w] = 1;
    }
}

__global__ void k_check(State s, double flatness, double lnf_final)
{
    check_window(s, blockIdx.x, flatness, lnf_final);
}

// tab[b] = (instance, window); prm[instance] = (flatness, ln f_final)
__global__ void k_check_batch(const State *__restrict__ states, const int2 *__restrict__ tab,
                              const double2 *__restrict__ prm)
{
    const int2 t = tab[blockIdx.x];
    const State s = states[t.x];
    const double2 p = prm[t.x];
    check_window(s, t.y, p.x, p.y);
}

cudaError_t launch_check_batch(const State *states, const int2 *tab, int n, const double2 *prm,
                               cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_check_batch<<<n, 512, 0, st>>>(states, tab, prm);
    return cudaGetLastError();
}

cudaError_t launch_check(const State &s, double flatness, double lnf_final, cudaStream_t st)
{
    k_check<<<s.h, 512, 0, st>>>(s, flatness, lnf_final);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Replica exchange (Eq. 1) between windows (w, w+1), w = round mod 2.  One warp per pair;
// lane 0 draws the partner permutation and the decisions (m is small), the swap itself
// exchanges configuration indices and bins.
// ---------------------------------------------------------------------------------------
// Partner permutation of the exchange of pair (gw, gw+1) in round rd (global window index gw):
// Fisher-Yates from Philox draws (i, rd, gw, swap tag), i = m-1 .. 1.  One warp; perm in shared
// memory, valid after the call for every lane.
__device__ __forceinline__ void exchange_perm(const State &s, int gw, long long rd, int *perm, int *draw)
{
    const int lane = threadIdx.x & 31, m = s.m;
    const uint32_t tag = (s.inst << 8) | TAG_SWAP;
    for (int i = lane; i < m; i += 32) {
        perm[i] = i;
        if (i >= 1) {
            const u32x4 r = philox((uint32_t)i, (uint32_t)rd, (uint32_t)gw, tag, s.key0, s.key1);
            draw[i] = (int)mulhi(r.x, (uint32_t)(i + 1));
        }
    }
    __syncwarp();
    if (lane == 0)
        for (int i = m - 1; i >= 1; --i) {
            const int j = draw[i];
            const int t = perm[i];
            perm[i] = perm[j];
            perm[j] = t;
        }
    __syncwarp();
}

// Accept decision of Eq. (1) for partner pair i: ln P >= 0 or ln u < ln P, u from Philox
// (m + i, rd, gw, swap tag).
__device__ __forceinline__ bool exchange_accept(const State &s, int gw, long long rd, int i, double lnP)
{
    if (lnP >= 0.0) return true;
    const u32x4 r = philox((uint32_t)(s.m + i), (uint32_t)rd, (uint32_t)gw, (s.inst << 8) | TAG_SWAP,
                           s.key0, s.key1);
    return lnu64(r.x) < lnP;
}

__device__ __forceinline__ void swap_pair(const State &s, const int pair)
{
    // one warp per window pair: the permutation's random draws and the m exchange decisions
    // are lane-parallel (each decision touches its own two walker slots); only the
    // Fisher-Yates swaps themselves run in order.  Pairs (w, w+1) with the global window
    // index w0 + w of the parity of the round.
    if (s.status->done) return;
    const long long rd = s.status->round;
    const int w = 2 * pair + (int)((rd + s.w0) & 1);
    if (w + 1 >= s.h) return;
    const int lane = threadIdx.x & 31;
    const int m = s.m, W = s.W;
    __shared__ int perm[MAX_M];
    __shared__ int draw[MAX_M];
    exchange_perm(s, s.w0 + w, rd, perm, draw);
    const int loA = s.lo[w], hiA = s.hi[w], loB = s.lo[w + 1], hiB = s.hi[w + 1];
    unsigned acc = 0;
    for (int i = lane; i < m; i += 32) {
        const int a = w * m + i, b = (w + 1) * m + perm[i];
        const int kx = s.k[a], ky = s.k[b];
        if (kx < loB || kx > hiB || ky < loA || ky > hiA) continue;
        const double *ga = s.lng + (size_t)a * W, *gb = s.lng + (size_t)b * W;
        const double lnP = __dadd_rn(__dsub_rn(ga[kx - loA], ga[ky - loA]),
                                     __dsub_rn(gb[ky - loB], gb[kx - loB]));
        if (exchange_accept(s, s.w0 + w, rd, i, lnP)) {
            const int t = s.cfg[a];
            s.cfg[a] = s.cfg[b];
            s.cfg[b] = t;
            s.k[a] = ky;
            s.k[b] = kx;
            ++acc;
        }
    }
    acc = __reduce_add_sync(FULL, acc);
    if (lane == 0) {
        s.swap_att[w] += (unsigned long long)m;
        s.swap_acc[w] += acc;
    }
}

__global__ void k_swap(State s) { swap_pair(s, blockIdx.x); }

// tab[b] = (instance, pair index)
__global__ void k_swap_batch(const State *__restrict__ states, const int2 *__restrict__ tab)
{
    const int2 t = tab[blockIdx.x];
    const State s = states[t.x];
    swap_pair(s, t.y);
}

cudaError_t launch_swap_batch(const State *states, const int2 *tab, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_swap_batch<<<n, 32, 0, st>>>(states, tab);
    return cudaGetLastError();
}

cudaError_t launch_swap(const State &s, cudaStream_t st)
{
    if (s.h < 2) return cudaSuccess;
    k_swap<<<(s.h + 1) / 2, 32, 0, st>>>(s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Window-sharded runs: the exchange of the pair that straddles a shard boundary (Eq. 1).
// Each shard runs its windows' rounds as usual; for the pair (gw, gw+1) across the boundary,
// the shard of gw (side 1, its last window) and the shard of gw+1 (side 0, its first window)
// trade, after the round, their walkers' bins, their half of ln P, and the lattices of the
// accepted pairs.  Both sides draw the same permutation and the same random numbers, and add
// the halves in the same order as the single-device exchange, so every decision is the same.
// The round whose exchange this is has just ended: rd = round counter - 1.  One warp each.
// ---------------------------------------------------------------------------------------
struct BndPair {
    int lw, gw;   // local window on this side, global index of the pair's lower window
    long long rd; // round of the exchange
    bool active;  // the pair exchanges in this round
};

__device__ __forceinline__ BndPair bnd_pair(const State &s, int side)
{
    BndPair b;
    b.lw = side ? s.h - 1 : 0;
    b.gw = side ? s.w0 + s.h - 1 : s.w0 - 1;
    b.rd = s.status->round - 1;
    b.active = b.rd >= 0 && ((b.rd - b.gw) & 1) == 0;
    return b;
}

__global__ void k_bnd_bins(State s, int side, int *bins)
{
    const int lw = side ? s.h - 1 : 0;
    for (int i = threadIdx.x; i < s.m; i += blockDim.x) bins[i] = s.k[lw * s.m + i];
}

__global__ void k_bnd_half(State s, int side, int plo, int phi, const int *pbins, double *half)
{
    __shared__ int perm[MAX_M];
    __shared__ int draw[MAX_M];
    const BndPair b = bnd_pair(s, side);
    const int lane = threadIdx.x & 31, m = s.m;
    if (!b.active) {
        for (int i = lane; i < m; i += 32) half[i] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    exchange_perm(s, b.gw, b.rd, perm, draw);
    const int lo = s.lo[b.lw], hi = s.hi[b.lw];
    for (int i = lane; i < m; i += 32) {
        double v = __longlong_as_double(0x7ff8000000000000LL); // NaN: the pair cannot exchange
        if (side) { // own walker i of the lower window holds X
            const int a = b.lw * m + i;
            const int kx = s.k[a], ky = pbins[perm[i]];
            const double *g = s.lng + (size_t)a * s.W;
            if (kx >= plo && kx <= phi && ky >= lo && ky <= hi) v = __dsub_rn(g[kx - lo], g[ky - lo]);
        } else { // own walker perm[i] of the upper window holds Y
            const int a = b.lw * m + perm[i];
            const int kx = pbins[i], ky = s.k[a];
            const double *g = s.lng + (size_t)a * s.W;
            if (kx >= lo && kx <= hi && ky >= plo && ky <= phi) v = __dsub_rn(g[ky - lo], g[kx - lo]);
        }
        half[i] = v;
    }
}

__global__ void k_bnd_decide(State s, int side, const double *half, const double *phalf, uint8_t *acc,
                             int8_t *lat_out)
{
    __shared__ int perm[MAX_M];
    __shared__ int draw[MAX_M];
    const BndPair b = bnd_pair(s, side);
    const int lane = threadIdx.x & 31, m = s.m;
    if (!b.active) {
        for (int i = lane; i < m; i += 32) acc[i] = 0;
        return;
    }
    exchange_perm(s, b.gw, b.rd, perm, draw);
    unsigned na = 0;
    for (int i = lane; i < m; i += 32) {
        const double lower = side ? half[i] : phalf[i], upper = side ? phalf[i] : half[i];
        const bool ok = lower == lower && upper == upper &&
                        exchange_accept(s, b.gw, b.rd, i, __dadd_rn(lower, upper));
        acc[i] = ok ? 1 : 0;
        na += ok;
    }
    na = __reduce_add_sync(FULL, na);
    __syncwarp();
    // the lattices this side hands over (read before the partner's arrive)
    for (int i = 0; i < m; ++i) {
        if (!acc[i]) continue;
        const int slot = b.lw * m + (side ? i : perm[i]);
        const int8_t *src = s.spins + (size_t)s.cfg[slot] * s.spin_stride;
        for (int j = lane; j < s.N; j += 32) lat_out[(size_t)i * s.N + j] = src[j];
    }
    if (side && lane == 0) { // the counters of pair gw live with its lower window
        s.swap_att[b.lw] += (unsigned long long)m;
        s.swap_acc[b.lw] += na;
    }
}

__global__ void k_bnd_import(State s, int side, const int *pbins, const uint8_t *acc, const int8_t *plat)
{
    __shared__ int perm[MAX_M];
    __shared__ int draw[MAX_M];
    const BndPair b = bnd_pair(s, side);
    const int lane = threadIdx.x & 31, m = s.m;
    if (!b.active) return;
    exchange_perm(s, b.gw, b.rd, perm, draw);
    for (int i = 0; i < m; ++i) {
        if (!acc[i]) continue;
        const int slot = b.lw * m + (side ? i : perm[i]);
        int8_t *dst = s.spins + (size_t)s.cfg[slot] * s.spin_stride;
        for (int j = lane; j < s.N; j += 32) dst[j] = plat[(size_t)i * s.N + j];
        if (lane == 0) s.k[slot] = side ? pbins[perm[i]] : pbins[i];
    }
}

cudaError_t launch_bnd_bins(const State &s, int side, int *bins, cudaStream_t st)
{
    k_bnd_bins<<<1, 128, 0, st>>>(s, side, bins);
    return cudaGetLastError();
}

cudaError_t launch_bnd_half(const State &s, int side, int plo, int phi, const int *pbins, double *half,
                            cudaStream_t st)
{
    k_bnd_half<<<1, 32, 0, st>>>(s, side, plo, phi, pbins, half);
    return cudaGetLastError();
}

cudaError_t launch_bnd_decide(const State &s, int side, const double *half, const double *phalf,
                              uint8_t *acc, int8_t *lat_out, cudaStream_t st)
{
    k_bnd_decide<<<1, 32, 0, st>>>(s, side, half, phalf, acc, lat_out);
    return cudaGetLastError();
}

cudaError_t launch_bnd_import(const State &s, int side, const int *pbins, const uint8_t *acc,
                              const int8_t *plat, cudaStream_t st)
{
    k_bnd_import<<<1, 32, 0, st>>>(s, side, pbins, acc, plat);
    return cudaGetLastError();
}

__device__ __forceinline__ void round_end(const State &s)
{
    if (s.status->done) return;
    s.status->round += 1;
    int all = !s.production;
    for (int w = 0; w < s.h; ++w) all &= s.finished[w];
    if (all) s.status->done = 1;
}

__global__ void k_round_end(State s) { round_end(s); }

__global__ void k_round_end_batch(const State *__restrict__ states, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) round_end(states[i]);
}

cudaError_t launch_round_end_batch(const State *states, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_round_end_batch<<<(n + 63) / 64, 64, 0, st>>>(states, n);
    return cudaGetLastError();
}

cudaError_t launch_round_end(const State &s, cudaStream_t st)
{
    k_round_end<<<1, 1, 0, st>>>(s);
    return cudaGetLastError();
}

__global__ void k_set_done(State s)
{
    int all = !s.production;
    for (int w = 0; w < s.h; ++w) all &= s.finished[w];
    s.status->done = all;
}

cudaError_t launch_set_done(const State &s, cudaStream_t st)
{
    k_set_done<<<1, 1, 0, st>>>(s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Joining (Sec. 3, Eq. 2).
// ---------------------------------------------------------------------------------------
__global__ void k_window_mean(State s, double *out)
{
    const int w = blockIdx.x, nb = s.hi[w] - s.lo[w] + 1;
    for (int b = threadIdx.x; b < s.W; b += blockDim.x) {
        double v = 0.0;
        if (b < nb) {
            double acc = 0.0;
            for (int i = 0; i < s.m; ++i) acc = __dadd_rn(acc, s.lng[(size_t)(w * s.m + i) * s.W + b]);
            v = __ddiv_rn(acc, (double)s.m);
        }
        out[(size_t)w * s.W + b] = v;
    }
}

cudaError_t launch_window_mean(const State &s, double *out, cudaStream_t st)
{
    k_window_mean<<<s.h, 256, 0, st>>>(s, out);
    return cudaGetLastError();
}

// beta by the 5-point (npts 5) or 3-point stencil at window-local bin b; 0 if not defined.
__device__ int stencil_beta(const double *l, const uint8_t *v, int nb, int b, int step, int npts,
                            double de, double *beta)
{
    if (npts == 5) {
        if (b - 2 * step < 0 || b + 2 * step >= nb) return 0;
        if (!(v[b - 2 * step] && v[b - step] && v[b + step] && v[b + 2 * step])) return 0;
        const double num = __dadd_rn(
            __dsub_rn(__dadd_rn(-l[b + 2 * step], __dmul_rn(8.0, l[b + step])),
                      __dmul_rn(8.0, l[b - step])),
            l[b - 2 * step]);
        *beta = __ddiv_rn(num, __dmul_rn(__dmul_rn(12.0, de), (double)step));
        return 1;
    }
    if (b - step < 0 || b + step >= nb) return 0;
    if (!(v[b - step] && v[b + step])) return 0;
    *beta = __ddiv_rn(__dsub_rn(l[b + step], l[b - step]),
                      __dmul_rn(__dmul_rn(2.0, de), (double)step));
    return 1;
}

// Block-wide argmin of (value, key): smaller value, ties -> smaller key.
__device__ void block_argmin(double &v, int &key)
{
    __shared__ double sv[32];
    __shared__ int sk[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(FULL, v, o);
        const int ok = __shfl_xor_sync(FULL, key, o);
        if (ov < v || (ov == v && ok < key)) {
            v = ov;
            key = ok;
        }
    }
    if (lane == 0) {
        sv[wid] = v;
        sk[wid] = key;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        v = lane < nw ? sv[lane] : INFINITY;
        key = lane < nw ? sk[lane] : 0x7fffffff;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(FULL, v, o);
            const int ok = __shfl_xor_sync(FULL, key, o);
            if (ov < v || (ov == v && ok < key)) {
                v = ov;
                key = ok;
            }
        }
        if (lane == 0) {
            sv[0] = v;
            sk[0] = key;
        }
    }
    __syncthreads();
    v = sv[0];
    key = sk[0];
    __syncthreads();
}

__device__ double block_reduce_max(double v)
{
    __shared__ double sv[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_max(v);
    if (lane == 0) sv[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sv[lane] : -INFINITY;
        v = warp_max(v);
        if (lane == 0) sv[0] = v;
    }
    __syncthreads();
    v = sv[0];
    __syncthreads();
    return v;
}

__device__ double block_reduce_sum(double v)
{
    __shared__ double sv[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0) sv[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sv[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (lane == 0) sv[0] = v;
    }
    __syncthreads();
    v = sv[0];
    __syncthreads();
    return v;
}

// One CTA: joins are found pair by pair (each depends on the previous one); the stencils
// and the argmin over the overlap are block-parallel.
__global__ void k_stitch(State s, const double *mean, double de, int step, int norm, double target,
                         double *out, int *joins, int *ok, int B)
{
    const int W = s.W;
    __shared__ double shift_s;
    __shared__ int prev_s, fail_s;
    for (int b = threadIdx.x; b <= B; b += blockDim.x) out[b] = -INFINITY;
    __syncthreads();
    {
        const int lo0 = s.lo[0], hi0 = s.hi[0];
        for (int b = lo0 + (int)threadIdx.x; b <= hi0; b += blockDim.x)
            if (s.mask[b - lo0]) out[b] = mean[b - lo0];
    }
    if (threadIdx.x == 0) {
        shift_s = 0.0;
        prev_s = -1;
        fail_s = 0;
    }
    __syncthreads();
    for (int w = 0; w + 1 < s.h; ++w) {
        const double *la = mean + (size_t)w * W, *lb = mean + (size_t)(w + 1) * W;
        const uint8_t *va = s.mask + (size_t)w * W, *vb = s.mask + (size_t)(w + 1) * W;
        const int loa = s.lo[w], hia = s.hi[w], lob = s.lo[w + 1], hib = s.hi[w + 1];
        const int nba = hia - loa + 1, nbb = hib - lob + 1;
        const int prev = prev_s;
        int kj = -1;
        for (int npts = 5; npts >= 3 && kj < 0; npts -= 2) {
            double best = INFINITY;
            int bk = 0x7fffffff;
            for (int k = lob + (int)threadIdx.x; k <= hia; k += blockDim.x) {
                if (k <= prev || !va[k - loa] || !vb[k - lob]) continue;
                double ba, bb;
                if (!stencil_beta(la, va, nba, k - loa, step, npts, de, &ba)) continue;
                if (!stencil_beta(lb, vb, nbb, k - lob, step, npts, de, &bb)) continue;
                const double db = fabs(__dsub_rn(ba, bb));
                if (db < best || (db == best && k < bk)) {
                    best = db;
                    bk = k;
                }
            }
            block_argmin(best, bk);
            if (best < INFINITY) kj = bk;
        }
        if (kj < 0) { // nearest bin valid in both to the overlap midpoint, ties -> smaller
            const int mid2 = lob + hia;
            double bd = INFINITY;
            int bk = 0x7fffffff;
            for (int k = lob + (int)threadIdx.x; k <= hia; k += blockDim.x) {
                if (k <= prev || !va[k - loa] || !vb[k - lob]) continue;
                const double d = fabs((double)(2 * k - mid2));
                if (d < bd || (d == bd && k < bk)) {
                    bd = d;
                    bk = k;
                }
            }
            block_argmin(bd, bk);
            if (bd < INFINITY) kj = bk;
        }
        if (kj < 0) {
            if (threadIdx.x == 0) fail_s = 1;
            break;
        }
        if (threadIdx.x == 0) {
            shift_s = __dsub_rn(__dadd_rn(la[kj - loa], shift_s), lb[kj - lob]);
            joins[w] = kj;
            prev_s = kj;
        }
        __syncthreads();
        const double sh = shift_s;
        for (int b = max(kj, lob) + (int)threadIdx.x; b <= hib; b += blockDim.x)
            out[b] = vb[b - lob] ? __dadd_rn(lb[b - lob], sh) : -INFINITY;
        __syncthreads();
    }
    __syncthreads();
    if (fail_s) {
        if (threadIdx.x == 0) *ok = 0;
        return;
    }
    if (norm == 0) {
        double mx = -INFINITY;
        for (int b = threadIdx.x; b <= B; b += blockDim.x) mx = fmax(mx, out[b]);
        mx = block_reduce_max(mx);
        double sum = 0.0;
        for (int b = threadIdx.x; b <= B; b += blockDim.x)
            if (out[b] > -INFINITY) sum += exp(out[b] - mx);
        sum = block_reduce_sum(sum);
        const double cst = (mx + log(sum)) - target;
        for (int b = threadIdx.x; b <= B; b += blockDim.x)
            if (out[b] > -INFINITY) out[b] -= cst;
    } else {
        int b0 = 0x7fffffff;
        double dummy = 0.0;
        for (int b = threadIdx.x; b <= B; b += blockDim.x)
            if (out[b] > -INFINITY && b < b0) b0 = b;
        block_argmin(dummy, b0);
        if (b0 > B) {
            if (threadIdx.x == 0) *ok = 0;
            return;
        }
        const double cst = __dsub_rn(out[b0], target);
        __syncthreads();
        for (int b = threadIdx.x; b <= B; b += blockDim.x)
            if (out[b] > -INFINITY) out[b] = __dsub_rn(out[b], cst);
    }
    if (threadIdx.x == 0) *ok = 1;
}

cudaError_t launch_stitch(const State &s, const double *mean, double de, int step, int norm,
                          double target, double *out, int *joins, int *ok, int B, cudaStream_t st)
{
    k_stitch<<<1, 256, 0, st>>>(s, mean, de, step, norm, target, out, joins, ok, B);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Diagnostics.
// ---------------------------------------------------------------------------------------
__global__ void k_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const u32x4 r = philox(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3],
                           key[2 * i], key[2 * i + 1]);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

cudaError_t launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n,
                          cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_philox<<<(n + 255) / 256, 256, 0, st>>>(ctr, key, out, n);
    return cudaGetLastError();
}

__global__ void k_lnu(const uint32_t *w, double *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = lnu64(w[i]);
}

cudaError_t launch_lnu(const uint32_t *w, double *out, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_lnu<<<(n + 255) / 256, 256, 0, st>>>(w, out, n);
    return cudaGetLastError();
}

__device__ __forceinline__ void atomic_max_pos(double *addr, double v)
{
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

__global__ void k_lnu_bound(uint64_t begin, uint64_t end, double *max_err, unsigned long long *n_bad)
{
    double mx = 0.0;
    unsigned long long bad = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = begin + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < end; x += stride) {
        const uint32_t w = (uint32_t)x;
        const double e = lnu64(w);
        const double f = (double)lnu32(w);
        mx = fmax(mx, fabs(f - e));
        bad += (e >= 0.0);
    }
    mx = warp_max(mx);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(FULL, bad, o);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_pos(max_err, mx);
        if (bad) atomicAdd(n_bad, bad);
    }
}

cudaError_t launch_lnu_bound(uint64_t begin, uint64_t end, double *max_err,
                             unsigned long long *n_bad, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(max_err, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(n_bad, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (end <= begin) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_lnu_bound<<<sms * 8, 256, 0, st>>>(begin, end, max_err, n_bad);
    return cudaGetLastError();
}

__global__ void k_seqadd(const double *x, const double *f, const uint32_t *c, double *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = seqadd(x[i], f[i], c[i]);
}

cudaError_t launch_seqadd(const double *x, const double *f, const uint32_t *c, double *out,
                          int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_seqadd<<<(n + 127) / 128, 128, 0, st>>>(x, f, c, out, n);
    return cudaGetLastError();
}

} // namespace rewl

namespace rewl {

// ---------------------------------------------------------------------------------------
// Canonical averages from ln g (Eqs. 6-7): one CTA per temperature; u = <E>/N,
// c = <(E - <E>)^2> / (N T^2), weights g(E) e^{-E/T} taken relative to their maximum.
// ---------------------------------------------------------------------------------------
__global__ void k_thermo(const double *__restrict__ lng, int B, int model, int N,
                         const double *__restrict__ Ts, double *__restrict__ U,
                         double *__restrict__ Cv)
{
    const double T = Ts[blockIdx.x];
    auto energy = [&](int b) { return -2.0 * N + (model == 0 ? 4.0 * b : (double)b); };
    double mx = -INFINITY;
    for (int b = threadIdx.x; b <= B; b += blockDim.x)
        if (lng[b] > -INFINITY) mx = fmax(mx, lng[b] - energy(b) / T);
    mx = block_reduce_max(mx);
    double s0 = 0.0, s1 = 0.0;
    for (int b = threadIdx.x; b <= B; b += blockDim.x)
        if (lng[b] > -INFINITY) {
            const double w = exp(lng[b] - energy(b) / T - mx);
            s0 += w;
            s1 += w * energy(b);
        }
    s0 = block_reduce_sum(s0);
    s1 = block_reduce_sum(s1);
    const double e1 = s1 / s0;
    double s2 = 0.0;
    for (int b = threadIdx.x; b <= B; b += blockDim.x)
        if (lng[b] > -INFINITY) {
            const double w = exp(lng[b] - energy(b) / T - mx);
            const double de = energy(b) - e1;
            s2 += w * de * de;
        }
    s2 = block_reduce_sum(s2);
    if (threadIdx.x == 0) {
        U[blockIdx.x] = e1 / N;
        Cv[blockIdx.x] = s2 / s0 / ((double)N * T * T);
    }
}

cudaError_t launch_thermo(const double *lng, int model, int L, const double *T, int nT, double *U,
                          double *C, cudaStream_t st)
{
    if (nT <= 0) return cudaSuccess;
    const int N = L * L, B = model == 0 ? N : 2 * N;
    k_thermo<<<nT, 256, 0, st>>>(lng, B, model, N, T, U, C);
    return cudaGetLastError();
}

} // namespace rewl

namespace rewl {

// Window means of the saved fragments leaving walker j out (walker order), [h][W].
__global__ void k_loo_mean(State s, int j, double *out)
{
    const int w = blockIdx.x, nb = s.hi[w] - s.lo[w] + 1;
    for (int b = threadIdx.x; b < s.W; b += blockDim.x) {
        double v = 0.0;
        if (b < nb) {
            double acc = 0.0;
            for (int i = 0; i < s.m; ++i)
                if (i != j) acc = __dadd_rn(acc, s.frag[(size_t)(w * s.m + i) * s.W + b]);
            v = __ddiv_rn(acc, (double)(s.m - 1));
        }
        out[(size_t)w * s.W + b] = v;
    }
}

cudaError_t launch_loo_mean(const State &s, int j, double *out, cudaStream_t st)
{
    k_loo_mean<<<s.h, 256, 0, st>>>(s, j, out);
    return cudaGetLastError();
}

// err[b] = sqrt((m-1)/m sum_j (theta_j[b] - mean)^2); NaN where any theta_j is -inf.
__global__ void k_jack(const double *theta, int m, int B, double *err)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > B) return;
    double mean = 0.0;
    bool ok = true;
    for (int j = 0; j < m; ++j) {
        const double v = theta[(size_t)j * (B + 1) + b];
        ok = ok && v > -INFINITY;
        mean += v;
    }
    if (!ok) {
        err[b] = NAN;
        return;
    }
    mean /= m;
    double ss = 0.0;
    for (int j = 0; j < m; ++j) {
        const double d = theta[(size_t)j * (B + 1) + b] - mean;
        ss += d * d;
    }
    err[b] = sqrt((double)(m - 1) / m * ss);
}

cudaError_t launch_jack(const double *theta, int m, int B, double *err, cudaStream_t st)
{
    k_jack<<<(B + 256) / 256, 256, 0, st>>>(theta, m, B, err);
    return cudaGetLastError();
}

} // namespace rewl
