/*
 * rewl.h -- C ABI of the GB300 (sm_103a) replica-exchange Wang-Landau library.
 *
 * Method: Li, Vogel, Wuest, Landau, "A new paradigm for petascale Monte Carlo
 * simulation: Replica exchange Wang-Landau sampling", arXiv:1402.2328.
 *
 * Conventions
 *   - Every int-returning function returns REWL_OK (0) or a negative REWL_ERR_* code;
 *     rewl_last_error() gives a message.  Nothing throws across this boundary.
 *   - Host pointers ("host") are caller-owned and only read or written during the call.
 *     Device pointers ("device") are caller-owned CUDA allocations on the current device;
 *     the call only enqueues work on the given stream.
 *   - A handle owns its device state (cudaMalloc'd in rewl_create, freed in rewl_destroy)
 *     and enqueues all work on the stream given by rewl_set_stream (default: the legacy
 *     default stream).  A handle is not thread safe.
 *   - Lattices: 2 <= L <= 255 and the move kernel's shared memory (3 bytes per site plus
 *     about 8.1 bytes per window bin) must fit one CTA (227 KB).
 *   - Models: model = 0 is the 2D Ising model E = -sum_<ij> s_i s_j (J = 1, s = +-1);
 *     model = q >= 2 is the q-state Potts model E = -sum_<ij> delta(s_i, s_j).  L x L
 *     square lattice with periodic boundaries, N = L*L sites, spins stored as int8.
 *   - Energy bins: k counts unsatisfied bonds.  Ising: k = (E + 2N)/4 in [0, N] (B = N);
 *     Potts: k = E + 2N in [0, 2N] (B = 2N).  ln g arrays over all bins have B+1 entries.
 */
#ifndef REWL_H
#define REWL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define REWL_OK 0
#define REWL_ERR_INVALID_ARG (-1)
#define REWL_ERR_CUDA (-2)
#define REWL_ERR_TIMEOUT (-3)
#define REWL_ERR_NOT_CONVERGED (-4)
#define REWL_ERR_BUFFER_TOO_SMALL (-5)
#define REWL_ERR_PREP (-6)
#define REWL_ERR_STATE (-7)
#define REWL_ERR_IO (-8)

/* rewl_run status */
#define REWL_STATUS_RUNNING 0
#define REWL_STATUS_DONE 1    /* every window reached ln f < ln f_final (Sec. 2, end)   */
#define REWL_STATUS_BUDGET 2  /* max_rounds or max_seconds used up first                  */
#define REWL_STATUS_ABORTED 3 /* rewl_abort() was called                                   */

typedef struct rewl_s *rewl_t;

/*
 * rewl_create -- one REWL simulation (Sec. 2): the bin range [0, B] is split into `windows`
 * equal-size windows with overlap fraction `overlap` (Fig. 1a); every window has
 * `walkers_per_window` independent WL walkers with their own ln g(E) (float64) and H(E)
 * (uint32).  The walk stops when every window reached ln f < lnf_final (f_final, Sec. 2);
 * a walker's histogram is flat when min H >= flatness * mean H over the window's visited
 * bins.  Window layout: o = 0.75 uses W = 4B/(h+3), lo_k = round(kB/(h+3)),
 * hi_k = round((k+4)B/(h+3)), hi_{h-1} = B; other o use round(k s), round(k s + W) with
 * W = B/(1+(h-1)(1-o)), s = (1-o) W.  Adjacent windows must overlap, else INVALID_ARG.
 * Defaults: seed 0, ln f_init = 1, swap interval 10^4 moves, prep budget 100 sweeps.
 * lnf_final < 2^-32 is refused (INVALID_ARG): the move kernel keeps ln g as an integer multiple
 * of 2^-32 and could not add a smaller ln f.  *out receives the handle.  Allocates device memory on the current device.
 */
int rewl_create(rewl_t *out, int model, int L, int windows, double overlap,
                int walkers_per_window, double lnf_final, double flatness);

/*
 * rewl_set_param -- before rewl_init.  Keys: "lnf_init" (ln f of the first iteration,
 * default 1; 2^-32 <= lnf_init < 2^20), "interval" (WL moves per walker between two flatness
 * checks and replica exchange attempts, Sec. 2; default 10000; at most 10^8), where
 * interval * lnf_init must stay below 2^30 (the range of the move kernel's ln g shadow); "prep_budget" (sweeps allowed to bring a
 * walker into its window, default 100), "instance" (0..2^24-1, enters the random
 * stream, default 0), "graph_rounds" (rounds per CUDA-graph replay, default 32; 0 = no
 * graph), "walkers_per_block" (warps per CTA of the move kernel; 0 = automatic: the power
 * of two covering walkers / SMs, at most 4), "check_all" (1 = decide every move with the
 * float64 path as well and count disagreements; diagnostic), "layout" (move kernel: 0 = one
 * warp per walker, the default; 1 = one thread per walker, for small lattices with many
 * walkers; both give identical results), "schedule" (0 = ln f halving,
 * f -> sqrt f, Sec. 2; 1 = the 1/t schedule of Belardinelli and Pereyra, an alternative
 * Sec. 2 allows: after a halving, once ln f < 1/t with t = moves per walker / visited bins
 * of the window, ln f = 1/t is recomputed at every check, where the m walkers' ln g are
 * averaged, without a flatness test), "profile" (1 = time move-kernel launches with CUDA
 * events, see rewl_kernel_time; may be changed at any time).  Unknown key or bad value:
 * INVALID_ARG.
 * Two keys may also be set after rewl_init (they drop the cached CUDA graph):
 * "production" (1 = rounds continue after every window finished: ln g and H stay frozen, the
 * walkers keep moving and exchanging, so every window performs a multicanonical walk with
 * weight 1/g_w(E) -- the production run of Sec. 3; rewl_run then ends only at max_rounds /
 * max_seconds; 0 = back to the normal end test) and "measure_em" (Ising only; 1 = allocate and
 * zero an (E, M) histogram of h x W x (N+1) uint32 and, after the moves of every round, count
 * each walker's (bin, number of up spins) in its window; 0 = free it; INVALID_ARG when
 * h W (N+1) > 2^30 or (B+1)(N+1) > 2^28).  Both
 * keys are meant for handles made by rewl_create: the batch runner (rewl_batch_*) does not
 * run the (E, M) measurement.
 */
int rewl_set_param(rewl_t r, const char *key, double value);

/* rewl_set_seed -- 64-bit seed; the Philox4x32-10 key is (seed low word, seed high word). */
int rewl_set_seed(rewl_t r, uint64_t seed);

/*
 * rewl_set_lng_init -- warm start (host, n == B+1 float64 values): every walker of every
 * window starts from lng_bins[lo..hi] instead of 0.  Before rewl_init.  Non-finite
 * values inside any window: INVALID_ARG.
 */
int rewl_set_lng_init(rewl_t r, const double *lng_bins, int n);

/*
 * rewl_set_windows -- replace the window layout (host, 2*h ints lo[0..h-1], hi[0..h-1];
 * lo[0] = 0, hi[h-1] = B, lo increasing, adjacent windows overlapping).  Before rewl_init.
 * Used for run-time balanced splitting (Fig. 1b) and learned window boundaries.
 */
int rewl_set_windows(rewl_t r, const int *lo_hi, int h);

/*
 * rewl_windows_equal -- the equal-size layout of Fig. 1a that rewl_create uses (the formula
 * given there), for B+1 bins, h windows and overlap fraction `overlap`, into host lo_hi (2*h
 * ints: lo[0..h-1] then hi[0..h-1]).  Host only, no device call.  INVALID_ARG when adjacent
 * windows would not overlap.
 */
int rewl_windows_equal(int B, int h, double overlap, int *lo_hi);

/*
 * rewl_windows_late_balanced -- windows balanced by the cost of the later WL iterations (Fig. 1b
 * names the first iteration; the footnote to it allows adapting the layout as the run
 * proceeds).  lo_hi (host, 2h ints) is the layout of a pre-run and rounds_per_iter[w] the
 * rounds its window w took per iteration over some later iterations (<= 0: not measured,
 * counted as the slowest).  Per window a = rounds per iteration / width^2 (a later iteration's
 * time grows about with the square of the width); every bin costs sqrt(a), averaged over the
 * windows covering it; lo_hi_out (2*h_new ints) = rewl_windows_balanced of that cost, so the
 * new windows have about equal a * width^2.  Host only.  INVALID_ARG for a bad layout or no
 * measured window.  (First-iteration balancing over-widens windows whose first iteration is
 * cheap: for q = 10 Potts L = 80 it left the high-energy windows 2-4 times wider than equal
 * ones and slower than before.)
 */
int rewl_windows_late_balanced(const int *lo_hi, int h, const double *rounds_per_iter, int B,
                               int h_new, double overlap, int *lo_hi_out);

/*
 * rewl_windows_balanced -- run-time balanced windows (Fig. 1b).  host cost[B+1] >= 0 is the
 * expected first-iteration work per bin; the h windows are the equal-size layout with overlap
 * `overlap` placed in the coordinate u(b) = (cumulative cost up to b) / (total cost), so every
 * window carries the same share of work (each kept >= 5 bins wide and overlapping the next).
 * Uniform cost gives the equal-size layout.  lo_hi: host, 2h ints (lo[], then hi[]).  Host only.
 */
int rewl_windows_balanced(const double *cost, int B, int h, double overlap, int *lo_hi);
/*
 * rewl_balanced_from_prerun -- the cost profile of a short pre-run with equal windows, after
 * every window finished its first iteration (field "first_iter_round" > 0): a bin's cost is the
 * mean, over the windows covering it, of (first-iteration rounds) / (window width); then
 * rewl_windows_balanced with h windows.  Use the result with rewl_set_windows on a new handle.
 */
int rewl_balanced_from_prerun(rewl_t pre, int h, double overlap, int *lo_hi);
/*
 * rewl_balanced_scaled -- the same cost profile carried over to the same model on an L x L
 * lattice (bins matched by energy per site, e = E/N), then rewl_windows_balanced with h windows
 * over that lattice's bins: window boundaries for a large lattice learned from a smaller one.
 */
int rewl_balanced_scaled(rewl_t pre, int L, int h, double overlap, int *lo_hi);

/* rewl_set_stream -- cudaStream_t (as void*) for all later work of this handle. */
int rewl_set_stream(rewl_t r, void *stream);

/*
 * rewl_init -- seeded random lattices (Ising +-1 / Potts 0..q-1 from Philox), then every
 * walker is driven into its window: single-site moves accepted iff the distance of k to
 * the window does not grow; after prep_budget sweeps a walker restarts once from the ground
 * state (all +1 / all 0), or from the checkerboard (+1/-1, 0/1) when 2 lo > B.  REWL_ERR_PREP if
 * a walker cannot reach its window.  Called by rewl_run if needed.
 */
int rewl_init(rewl_t r);

/*
 * rewl_run -- runs rounds until every window is finished, max_rounds rounds were done
 * (max_rounds < 0: no limit) or max_seconds passed (<= 0: no limit).  One round is, for
 * every walker, `interval` WL moves (accept iff ln u < ln g(E_old) - ln g(E_new), then
 * ln g(E) += ln f, H(E)++; Sec. 2), then the per-walker flatness test and, for windows
 * whose m walkers are all flat, the averaging of ln g over the m walkers, H = 0 and
 * ln f /= 2 (Sec. 2), then replica exchange between windows (w, w+1), w = round mod 2,
 * with acceptance min[1, g_i(E_X) g_j(E_Y) / (g_i(E_Y) g_j(E_X))] (Eq. 1).
 * *status (may be NULL) gets a REWL_STATUS_* value.  Blocks until the work is done.
 */
int rewl_run(rewl_t r, double max_seconds, long long max_rounds, int *status);

/* rewl_abort -- asks a running rewl_run (another thread) to stop after the current chunk. */
int rewl_abort(rewl_t r);

/*
 * rewl_step -- enqueues `rounds` rounds (as rewl_run performs them) on the handle's stream
 * and returns without waiting.  Rounds enqueued after every window finished do nothing.
 * rewl_init must have succeeded.  Errors raised on the device show up in the next
 * rewl_run / rewl_stats / rewl_get_state call.
 */
int rewl_step(rewl_t r, int rounds);

/*
 * rewl_kernel_time -- with parameter "profile" = 1, every move-kernel launch is bracketed
 * by CUDA events on the handle's stream; this returns the summed duration (ms) and the
 * number of timed launches since the last reset (waits for them), and resets if reset != 0.
 */
int rewl_kernel_time(rewl_t r, double *move_ms, long long *launches, int reset);

/*
 * rewl_get_lng -- ln g of one walker (walker >= 0) or the mean over the window's walkers
 * (walker = -1, the mean of Sec. 2 taken in walker order) for bins lo..hi of `window`.
 * out: host, cap >= hi-lo+1 float64; *lo, *hi (may be NULL) receive the window bounds.
 */
int rewl_get_lng(rewl_t r, int window, int walker, double *out, int cap, int *lo, int *hi);

/*
 * rewl_stitch -- joins the window means into one ln g over all B+1 bins (Sec. 3, Eq. 2):
 * beta(k) = d ln g/dE by the 5-point stencil (3-point if no 5-point bin, Fig. 2); for each
 * adjacent pair the join bin minimises |beta_w - beta_{w+1}| over the overlap (ties: the
 * smaller bin, always after the previous join; no stencil: the bin valid in both windows
 * nearest the overlap midpoint); window w+1 is shifted to agree at the join; bins below the
 * join come from the left, the rest from the right.  Unvisited bins are -INFINITY.
 * norm = 0: logsumexp = N ln q;  norm = 1: ln g(ground state) = ln q.
 * out: host, cap >= B+1.  joins: host, h-1 ints, or NULL.  Runs on the GPU.
 */
int rewl_stitch(rewl_t r, double *out, int cap, int norm, int *joins);

/*
 * rewl_jackknife -- statistical error of the joined ln g from the m walkers' fragments
 * (Sec. 3: resampling over the walkers): each walker's ln g just before its window's last
 * averaging is kept; for j = 1..m the windows' means without walker j are joined as in
 * rewl_stitch (same norm), and err[b] = sqrt((m-1)/m * sum_j (theta_j[b] - mean)^2), NaN where a
 * resample has no value.  Needs m >= 2 and every window finished.  err: host, cap >= B+1.
 */
int rewl_jackknife(rewl_t r, double *err, int cap, int norm);

/*
 * rewl_dims -- out (host, 8 ints): N, B, windows, walkers per window, W (row stride of
 * per-walker ln g / H arrays = widest window), q, L, model.
 */
int rewl_dims(rewl_t r, int *out);

/*
 * rewl_get_state / rewl_set_state -- raw state, by field name, copied to/from host
 * memory of exactly `bytes` bytes (BUFFER_TOO_SMALL otherwise).  Fields (nw = h*m):
 *   "spins" int8[nw][N] (lattice carried by each walker slot), "k" int32[nw],
 *   "lng" float64[nw][W], "H" uint32[nw][W], "step" uint64[nw] (WL attempts of the slot),
 *   "acc" uint64[nw] (accepted moves), "flat" uint8[nw], "lnf" float64[h], "iter" int32[h],
 *   "finished" uint8[h], "mask" uint8[h][W] (bins visited by the window), "swap_att"
 *   uint64[h], "swap_acc" uint64[h] (pair (w,w+1) at index w), "pstep" uint64[nw],
 *   "prep_restarts" int32[nw], "round" int64[1], "lo" int32[h], "hi" int32[h],
 *   "n_exact" uint64[1] (moves decided by the float64 path), "n_mismatch" uint64[1],
 *   "lng_mean" float64[h][W] (window means of ln g, walker order; computed on the GPU),
 *   "first_iter_round" int64[h] (rounds done when the window's first iteration ended, 0 if
 *   not yet: times `interval` it is the MC steps of Eq. (5)), "mode" uint8[h] (1: 1/t),
 *   "frag" float64[nw][W] (each walker's ln g just before its window's last averaging).
 * rewl_set_state accepts "spins", "k", "lng", "H", "step", "flat", "lnf" (each in [0, 2^20)),
 * "iter", "finished" (the run's done flag is re-evaluated), "mask", "mode" (0/1 flags) and
 * "round" (tests plant late-stage states with it); values outside those ranges are refused
 * with REWL_ERR_INVALID_ARG.
 */
int rewl_get_state(rewl_t r, const char *field, void *out, size_t bytes);
int rewl_set_state(rewl_t r, const char *field, const void *in, size_t bytes);

/*
 * Window-sharded runs (Sec. 2: walkers in different energy windows only meet in the exchange
 * of Eq. (1), between neighbouring windows).  A run over h_global windows is split into
 * shards of consecutive windows, one handle each (typically one per GPU); the handles' state
 * together equals that of one handle over all windows, round for round, bit for bit.
 *
 * rewl_set_shard -- before rewl_init, on a handle made by rewl_create with `windows` = the
 * number of windows of this shard: lo_hi (host, 2 h_global ints: lo[0..h-1] then hi[0..h-1])
 * is the global layout (lo[0] = 0, hi[h-1] = B, adjacent windows overlapping) and the shard
 * holds windows w_begin .. w_begin + windows - 1.  Random streams use global window and walker
 * indices.  A shard never ends a run by itself (it behaves as with "production" = 1): the
 * caller ends the run when every shard reports all its windows finished (rewl_stats).
 * INVALID_ARG for a bad layout or range; STATE after rewl_init.
 *
 * After every round (rewl_step(r, 1) on every shard), the pair of windows across each shard
 * boundary exchanges through four calls on each side and three transfers the caller makes
 * (any transport: NCCL, MPI, host copies).  side 1 = this shard's last window (the pair's
 * lower window), side 0 = its first window (the pair's upper window).  In a round where that
 * pair does not exchange (round parity) the calls are still made and change nothing.  All
 * buffers are device memory of the handle's device; work goes to the handle's stream:
 *   rewl_boundary_bins(side, bins)                    bins: out, m int32 (the side's walkers' bins)
 *     -> send bins to the partner shard, receive its bins as partner_bins
 *   rewl_boundary_half(side, partner_bins, half)      half: out, m float64 (this side's term of ln P
 *                                                     for each partner pair i; NaN: cannot exchange)
 *     -> send half, receive the partner's as partner_half
 *   rewl_boundary_decide(side, half, partner_half, accepted, lattices)
 *                                                     accepted: out, m uint8 (same on both sides);
 *                                                     lattices: out, m x N int8, the lattices this
 *                                                     side hands over (rows of accepted pairs)
 *     -> send lattices, receive the partner's as partner_lattices
 *   rewl_boundary_import(side, partner_bins, accepted, partner_lattices)
 * STATE if the handle is not an initialised shard; INVALID_ARG for a side without a neighbour.
 */
int rewl_set_shard(rewl_t r, const int *lo_hi, int h_global, int w_begin);
int rewl_boundary_bins(rewl_t r, int side, int *bins);
int rewl_boundary_half(rewl_t r, int side, const int *partner_bins, double *half);
int rewl_boundary_decide(rewl_t r, int side, const double *half, const double *partner_half,
                         uint8_t *accepted, int8_t *lattices);
int rewl_boundary_import(rewl_t r, int side, const int *partner_bins, const uint8_t *accepted,
                         const int8_t *partner_lattices);

/* Run statistics (Sec. 2 exchange acceptance; Eq. 5 step counts). */
typedef struct {
    long long rounds;            /* rounds executed */
    long long attempts;          /* WL attempts, all walkers */
    long long accepted;          /* accepted WL moves */
    long long swap_attempts;     /* replica-exchange attempts */
    long long swap_accepted;     /* accepted exchanges */
    long long exact_decisions;   /* moves decided by the float64 path */
    long long prep_restarts;     /* walkers restarted from the ordered state */
    int windows_finished;        /* windows with ln f < ln f_final */
    int min_iteration;           /* smallest completed-iteration count over windows */
    double max_lnf;              /* largest current ln f over windows */
    double seconds;              /* wall time spent in rewl_run */
} rewl_stats_t;
int rewl_stats(rewl_t r, rewl_stats_t *out);

/*
 * rewl_checkpoint / rewl_restore -- the whole state (lattices, bins, ln g, H, step
 * counters, flags, ln f, iterations, masks, 1/t modes, saved fragments, round, the production
 * switch and, when the (E, M) measurement is on, its histogram) to/from a binary file.  The
 * random stream is a function of the step counters, so a restored run continues bit for bit.
 * rewl_restore needs a handle created with the same parameters, including "schedule" (else
 * INVALID_ARG); it takes over the checkpoint's production switch and (E, M) measurement.
 */
int rewl_checkpoint(rewl_t r, const char *path);
int rewl_restore(rewl_t r, const char *path);

void rewl_destroy(rewl_t r);

/* Message for the last error of r (or of a failed rewl_create / free function if r = NULL). */
const char *rewl_last_error(rewl_t r);

/*
 * Joint density of states g(E, Q) with Q = magnetisation M of the Ising model (Sec. 3,
 * Eqs. 3-4).  Bins: k as in rewl_get_lng, j = number of up spins = (M + N)/2 in [0, N].
 *
 * rewl_get_hist_em -- the (E, M) histogram (host, bytes == h*W*(N+1)*4): [w][k - lo_w][j].
 * STATE if "measure_em" is off.
 */
int rewl_get_hist_em(rewl_t r, uint32_t *out, size_t bytes);
/*
 * rewl_stitch_em -- g(E, M) from the measured fragments: for every window w the fragment
 * S_w(k, j) = mean ln g_w(k) + ln H_w(k, j) - ln sum_j H_w(k, j) (absent where H_w = 0 or the bin
 * is unvisited), then rewl_join_em with dE = 4 per bin, dM = 2 per up spin, normalised to
 * sum g = 2^N.  out: host, n >= (B+1)(N+1) values, row-major [k][j], -INFINITY where absent.
 * joins: host, 2(h-1) ints (may be NULL).  Blocks until done.
 */
int rewl_stitch_em(rewl_t r, double *out, size_t n, int *joins);
/*
 * rewl_join_em -- joins 2D fragments (Sec. 3, Eqs. 3-4).  S: device, [h][W][N1] float64,
 * fragment w's row b is bin lo_w + b (rows past hi_w - lo_w ignored), -INFINITY = absent.
 * For each adjacent pair (w, w+1) the unit normals n = (dS/dE, dS/dQ, -1)/|.| (5-point stencil
 * along an axis where the four neighbours are present, else 3-point; de, dq = physical step per
 * bin and per j) are compared at every point of the overlap present in both with a normal in
 * both; the join point maximises n_w . n_(w+1) (ties: smallest bin, then smallest j; with no
 * such point: the point present in both nearest to the middle of the overlap rows).  Window
 * w+1 is shifted to agree there with the already shifted window w; the windows are merged in
 * order with Eq. (4): where both are present g = (g_i + g_j)/2.  out: device, (B+1) x N1,
 * normalised to logsumexp(out) = norm_target.  lo_hi: host, 2h ints (lo[], then hi[]; windows
 * as in rewl_set_windows).  joins: host, 2(h-1) ints (bin, j) or NULL.  NOT_CONVERGED when
 * two adjacent fragments share no point.  Scratch is allocated and freed inside; blocks.
 */
int rewl_join_em(const double *S, int h, int W, int B, int N1, const int *lo_hi, double de,
                 double dq, double norm_target, double *out, int *joins, void *stream);

/*
 * Batched instances.  Many independent REWL simulations (any mix of models, L, window
 * counts, walkers per window; each with its own seed and instance id) advanced together,
 * round by round: one move-kernel launch whose CTAs each serve up to `walkers_per_block`
 * walkers of one instance, then batched flatness/advance, exchange and round-end kernels,
 * rounds captured in CUDA graphs.  Every instance evolves bit for bit as it would alone with
 * rewl_create/rewl_run (same parameters, seed, instance id and interval).
 */
typedef struct rewl_batch_s *rewl_batch_t;
typedef struct {
    int model;              /* 0 = Ising, q >= 2 = q-state Potts */
    int L, windows, walkers_per_window;
    double overlap, lnf_final, flatness;
    double lnf_init;        /* <= 0: default 1 */
    uint64_t seed;
    int instance;           /* enters the random stream (0..2^24-1) */
} rewl_desc_t;

/* n instances (host array of descriptors), all with the same moves-per-round `interval`. */
int rewl_batch_create(rewl_batch_t *out, const rewl_desc_t *descs, int n, long long interval);
/* Keys: "walkers_per_block" (upper bound of warps per CTA, 0 = automatic),
 * "thread_layout_max_sites" (instances with at most this many sites run one thread per walker,
 * up to 32 x walkers_per_block walkers per CTA; 0 = none, the default), "graph_rounds",
 * "profile" (time the move kernel with events, rewl_batch_kernel_time), "check_all",
 * "prep_budget" (before init). */
int rewl_batch_set_param(rewl_batch_t b, const char *key, double value);
int rewl_batch_set_stream(rewl_batch_t b, void *stream);
/* Seeds and preps every instance (rewl_init) and builds the device tables. */
int rewl_batch_init(rewl_batch_t b);
/* Enqueue `rounds` rounds without waiting (rounds of finished instances do nothing). */
int rewl_batch_step(rewl_batch_t b, int rounds);
/* Run until every instance is done, max_rounds (< 0: no limit) or max_seconds (<= 0: none). */
int rewl_batch_run(rewl_batch_t b, double max_seconds, long long max_rounds, int *status);
/*
 * Autotuner.  First it times `rounds` rounds for every pair of a walkers-per-CTA bound in
 * {2, 4, 8, 16} and a thread-per-walker site limit in {0, 400, 1024, 1600} (which instances run
 * one thread per walker, hence how many windows of an instance share a CTA), and keeps the
 * fastest; then, with that layout, it times one CUDA-graph replay of each length in
 * {8, 32, 128} rounds (the kernel schedule between exchanges) and keeps the fastest.  The
 * trial rounds are ordinary rounds of the simulation (results do not depend on the launch
 * configuration).  best (may be NULL, 3 ints) gets walkers per CTA, site limit and graph
 * rounds; ms (may be NULL, REWL_BATCH_TUNE_CANDIDATES doubles) the milliseconds per round of
 * each candidate, index 4 * (site-limit index) + (walkers index), then the three graph
 * lengths; -1 for a site limit no instance falls under (the same layout as limit 0).
 */
#define REWL_BATCH_TUNE_CANDIDATES 19
int rewl_batch_autotune(rewl_batch_t b, int rounds, int *best, double *ms);
/* Instance i as a handle for the query calls (get_state, get_lng, stitch, stats,
 * checkpoint); owned by the batch: do not destroy it or run it on its own.  Before
 * rewl_batch_init, rewl_set_windows on it replaces the instance's window layout (e.g. run-time
 * balanced windows, Fig. 1b). */
int rewl_batch_instance(rewl_batch_t b, int i, rewl_t *out);
/* out (6 ints): instances, total walkers, CTAs of the move launch, warps per CTA,
 * thread-per-walker site limit, rounds per graph replay. */
int rewl_batch_info(rewl_batch_t b, int *out);
int rewl_batch_kernel_time(rewl_batch_t b, double *move_ms, long long *launches, int reset);
void rewl_batch_destroy(rewl_batch_t b);
const char *rewl_batch_last_error(rewl_batch_t b);

/*
 * rewl_replay -- n independent WL attempt sequences of T steps each, on caller state, with
 * caller-given random words instead of Philox (the move of Sec. 2 exactly as rewl_run
 * performs it, same kernel).  All pointers are device pointers:
 *   spins int8[n][N] (in/out), k int32[n] (in/out, must lie in [lo,hi]), lo/hi int32[n],
 *   lng float64[n][W] (in/out, window-local: index k-lo), H uint32[n][W] (in/out),
 *   lnf float64[n], frozen uint8[n] (1: no ln g/H update), words uint32[n][T][3]
 *   (w0 -> site, w1 -> Potts new state, w2 -> u = (w2 + 1/2) 2^-32),
 *   acc int32[n][T] and dk int32[n][T] (out: accepted flag and proposed bin change).
 * W >= max(hi-lo+1); a case with k outside [lo, hi], |ln g| >= 2^30, or (not frozen) ln f
 * outside [2^-32, 2^20) or max|ln g| + T ln f >= 2^30 (the range of the kernel's int64 ln g
 * shadow) makes the call fail with INVALID_ARG and leaves that case's state untouched.
 * stream: cudaStream_t or NULL.
 */
int rewl_replay(int model, int L, int n, int W, int T, void *spins, void *k, const void *lo,
                const void *hi, void *lng, void *H, const void *lnf, const void *frozen,
                const void *words, void *acc, void *dk, void *stream);

/*
 * Learned warm start.  A 3 -> 64 -> 64 -> 1 MLP (tanh, float32 weights) maps the features
 * (e = E/N in the Potts convention -- Ising energies mapped by E_P = (E_I - 2N)/2 --, q, 1/L)
 * of an energy bin to ln g(E)/N (g normalised to sum q^N).  It is trained on converged ln g of
 * small lattices and predicts a warm-start ln g for a larger one (rewl_set_lng_init); the run
 * then starts from a small ln f.  The paper has no counterpart; plain cold-start REWL stays the
 * fallback and the reference for its error.  All pointers are device pointers; stream may be NULL.
 * Parameter vector P (REWL_MLP_NPARAM floats): W1[64][3], b1[64], W2[64][64] (W2[i][j]: from
 * hidden-1 unit j to hidden-2 unit i), b2[64], W3[64], b3.  X: n x 3 features, T: n targets.
 */
#define REWL_MLP_NPARAM 4481
/* Y[i] = net(X[i]). */
int rewl_mlp_forward(const float *P, const float *X, float *Y, int n, void *stream);
/* floats of workspace rewl_mlp_grad / rewl_mlp_train need for n samples */
int rewl_mlp_workspace_floats(int n);
/* grad = d/dP of mean_i (net(X_i) - T_i)^2 (back-propagation; sums in sample order, so the
 * result does not depend on scheduling); *loss (device, may be NULL) = that mean. */
int rewl_mlp_grad(const float *P, const float *X, const float *T, int n, float *grad, float *loss,
                  float *work, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; t >= 1) on P with state m, v. */
int rewl_mlp_adam(float *P, const float *grad, float *m, float *v, int t, double lr, void *stream);
/* `steps` full-batch Adam steps (step numbers t0+1 ...); loss_out (may be NULL) gets the loss
 * before the last step.  grad: NPARAM floats; work: rewl_mlp_workspace_floats(n) floats. */
int rewl_mlp_train(float *P, const float *X, const float *T, int n, int steps, double lr, int t0,
                   float *m, float *v, float *grad, float *work, float *loss_out, void *stream);
/* Glorot-uniform weights from Philox4x32-10 keyed by seed, zero biases. */
int rewl_mlp_init(float *P, uint64_t seed, void *stream);
/* Training samples of one converged ln g (B+1 float64 values, -INFINITY = unvisited): one per
 * visited bin, in bin order, written to X (3 floats each) and T; *count (device int) = number. */
int rewl_mlp_samples(const double *lng, int model, int L, float *X, float *T, int *count,
                     void *stream);
/* lng[b] = N * net(e_b, q, 1/L) for the B+1 bins of lattice (model, L), float64. */
int rewl_mlp_predict(const float *P, int model, int L, double *lng, void *stream);
const char *rewl_mlp_last_error(void);

/*
 * rewl_thermo -- canonical averages from a density of states (Eqs. 6-7), k_B = 1: for each
 * temperature T[i], U[i] = <E>/N and C[i] = (<E^2> - <E>^2) / (N T[i]^2), the averages weighted
 * by g(E) e^{-E/T}.  lng: device, B+1 float64 (-INFINITY = unreachable bin); T, U, C: device,
 * nT float64.  Bin energies: Ising E = -2N + 4k, Potts E = -2N + k.
 */
int rewl_thermo(const double *lng, int model, int L, const double *T, int nT, double *U, double *C,
                void *stream);

/*
 * rewl_replay_static -- rewl_replay that allocates nothing.  The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc, e.g. code that draws all device
 * memory from its own pool (a framework's caching allocator holding most of the GPU), or
 * code that must not stall the device (rewl_replay's cudaFree of its per-call scratch waits
 * for the GPU).  Same arguments, results and errors as rewl_replay; the caller still owns
 * and passes every input and output.  The per-case scratch of the move kernel (step and
 * acceptance counters and the run status) lives instead in one fixed device array of the
 * library, sized for REWL_REPLAY_STATIC_MAX_N cases (about 256 KB, held on every GPU that
 * loads the library until the process exits); n > REWL_REPLAY_STATIC_MAX_N fails with
 * INVALID_ARG.  The first call on a device looks the array's device address up on that
 * device (cudaGetSymbolAddress); make that first call before any stream capture.  Every call
 * zeroes the part of the array it uses and then overwrites it, so the array keeps the last
 * call's contents, and calls whose work overlaps on the GPU (other streams, other threads)
 * race on it: serialise them.  The address is kept per device index for the life of the
 * process, so no call may follow a cudaDeviceReset of that device.
 */
#define REWL_REPLAY_STATIC_MAX_N 16384
int rewl_replay_static(int model, int L, int n, int W, int T, void *spins, void *k,
                       const void *lo, const void *hi, void *lng, void *H, const void *lnf,
                       const void *frozen, const void *words, void *acc, void *dk, void *stream);

/*
 * Diagnostics of the arithmetic the moves depend on (device pointers, stream or NULL):
 *   rewl_philox: out[i][0..3] = Philox4x32-10(ctr[i][0..3], key[i][0..1]) for i < n
 *     (Salmon et al., SC'11).
 *   rewl_lnu: out[i] = the float64 ln((w[i] + 1/2) 2^-32) that decides moves and exchanges.
 *   rewl_lnu_bound: over words w in [begin, end): max |screen(w) - lnu(w)| of the float32
 *     screening value into max_err (device, 1 float64, overwritten), and the count of words
 *     where the float64 value is >= 0 into n_bad (device, 1 uint64, overwritten).
 *   rewl_lnu_eps: the screening tolerance the move kernel assumes (host value).
 */
int rewl_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n, void *stream);
int rewl_lnu(const uint32_t *w, double *out, int n, void *stream);
int rewl_lnu_bound(uint64_t begin, uint64_t end, double *max_err, unsigned long long *n_bad,
                   void *stream);
double rewl_lnu_eps(void);
/* rewl_seqadd: out[i] = x[i] + f[i] + ... + f[i] (c[i] float64 additions, in order), device. */
int rewl_seqadd(const double *x, const double *f, const uint32_t *c, double *out, int n,
                void *stream);

#ifdef __cplusplus
}
#endif

#endif /* REWL_H */
