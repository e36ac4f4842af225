// Fused planner: everything between two update launches in one cooperative
// kernel (all blocks co-resident, separated by grid barriers whose waits are
// bounded):
//
//   A  front heights h(x) = 1 + highest occupied row of the bitmask (one warp
//      per 32-column word, one ballot per column), per-block Eq. 6 sums; one
//      block meanwhile works out n_s = floor(g M / rho_cell + carry) (Sec. II)
//      from the mass the update accumulated;
//   B  (every block, redundantly) the rear-wall rule (App. A, last paragraph)
//      with Eq. 6, the mass of the rows it freezes (n_s again if any), and
//      the candidate window of the growth mode;
//   C  the first candidates of the counter stream Philox (k, t, 1, sim), each
//      block a contiguous range: node, pair, rho* gathered from the nine
//      pre-stream slots, acceptance by the growth mode (Eq. 5 for density-
//      dependent growth), the block's accepted count;
//   D  draw ranks of the accepted candidates (block prefix over the other
//      blocks' counts); the first n_s are counted in an open-addressing table
//      keyed by (node, pair) and listed by rank (more candidates are drawn in
//      rounds if the first pass came up short);
//   E  per rank: the count of its (node, pair) if it was the first draw of
//      it (0 for repeats), and for the TMA-staged update one record in the
//      bucket of the CTA that owns its tile (that kernel adds count *
//      rho_cell/2 to the staged pre-stream slots; for the other update kernels
//      k_inject adds it to the stored populations right before the update);
//      the table is emptied again.
//
// Block 0 then writes the observables, commits the statistics of the step
// that just ran (its divisions were selected by the previous k_plan) and
// keeps the new selection's statistics pending.
#pragma once

#include "lbm_d2q7.cuh"
#include "lbm_kernels.cuh"
#include "lbm_tma.cuh"

namespace lbm {

constexpr int PLAN_NT = 512;
constexpr int PLAN_WARPS = PLAN_NT / 32;
constexpr int PLAN_R = 8; // candidates per thread in the first pass
// Grid barrier on a monotone arrival counter: a block's thread 0 adds one and
// waits until the counter reaches the next multiple of the grid size (the
// counter starts every launch at zero: the launch's last block out resets it,
// so successive launches may use different grids). The wait is bounded by
// `budget` clock cycles: on timeout ST_TIMEOUT is raised and later barriers
// no longer wait.
// `extra`: arrivals waited for beyond the grid (1 only in the failure-
// detection test, so that the wait runs out).
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// (G: the blocks of the grid that plan this simulation; with one block the
// barrier is the block's own.)
__device__ __forceinline__ void plan_grid_sync(DevScalars *sc, int *s_dead, int G, long long budget, int extra)
{
    __syncthreads();
    if (G == 1) return;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long g = (unsigned long long)G;
        const unsigned long long old = atomicAdd(&sc->bar_ctr, 1ull);
        const unsigned long long target = (old / g + 1ull) * g + (unsigned long long)extra;
        if (!*s_dead) {
            const long long t0 = clock64();
            while (ld_acquire_u64(&sc->bar_ctr) < target) {
                if (clock64() - t0 > budget) {
                    *s_dead = 1;
                    atomicOr(&sc->status, ST_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Block-wide sums / extrema of one value per thread (result on every thread).
__device__ __forceinline__ long long plan_block_sum(long long v, long long *s_ll)
{
    v = warp_sum_ll(v);
    if ((threadIdx.x & 31) == 0) s_ll[threadIdx.x >> 5] = v;
    __syncthreads();
    long long r = 0;
    for (int i = 0; i < PLAN_WARPS; ++i) r += s_ll[i];
    __syncthreads();
    return r;
}

// Exclusive block scan of one count per thread; *total gets the block sum.
__device__ __forceinline__ int plan_block_exscan(int v, int *total, int *s_i)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_i[warp] = incl;
    __syncthreads();
    int before = 0, all = 0;
    for (int i = 0; i < PLAN_WARPS; ++i) {
        const int c = s_i[i];
        before += i < warp ? c : 0;
        all += c;
    }
    __syncthreads();
    *total = all;
    return before + incl - v;
}

// The division of draw rank `rank`: merged in the table keyed by (node,
// pair) and counted at the rank of the pair's first draw (ev_count of a
// repeat stays 0; the counts were zeroed for this selection). The rank's list
// entry is the table slot if this draw was the first of its (node, pair),
// else -1. For the TMA-staged update, a first draw also gets its record and
// a place in its owner CTA's bucket (y_r: the rear wall of the coming step).
template <typename R, typename LT = Lat9>
__device__ __forceinline__ void plan_select(const SimDev &d, uint32_t key, int rank, size_t buf, int y_r)
{
    EventTable tb;
    tb.e = d.htab;
    tb.mask = (unsigned)d.hcap - 1u;
    int first;
    const int slot = table_insert(tb, key, rank, &first);
    d.hlist[rank] = slot;
    d.ev_key[buf + rank] = key;
    if (first >= 0) atomicAdd(&d.ev_count[buf + first], 1);
    if (d.inject_in_update) { // records for the TMA-staged update
        if (slot >= 0) {
            int owner;
            if constexpr (LT::Q == 9)
                owner = division_record<R>(d, rank, key, y_r);
            else
                owner = division_record7(d, rank, key, y_r);
            const int at = atomicAdd(&d.bucket_cnt[owner], 1);
            if (at < kBucketCap) d.bucket[owner * kBucketCap + at] = rank;
        } else {
            d.rec_owner[rank] = -1;
        }
    }
}

// Acceptance of a candidate (as `accept`, with the heights of this launch
// read from L2: other blocks wrote them before the last grid barrier).
template <typename S, typename LT = Lat9>
__device__ __forceinline__ bool plan_accept(const SimDev &d, const S *f, int y_r, const Candidate &c)
{
    using R = arith_t<S>;
    const R rs = rho_star<S, LT>(d, f, y_r, c.x, c.y);
    switch (d.growth_mode) {
    case GROW_BULK:
    case GROW_BAND: return rs >= rho_c_of<R>(d);
    case GROW_EDGE: return rs >= rho_c_of<R>(d) && (__ldcg(&d.heights[c.x]) - c.y) <= d.edge_depth;
    case GROW_DENSITY: return (double)rs > d.rho_c && u01(c.u) < 1.0 - (double)rs / d.rho0; // Eq. 5
    default: return false;
    }
}

// n_s = floor(g M / rho_cell + carry) (Sec. II) from the fixed-point active
// mass, and the carried fraction after it, in FP64 as the oracle. Also the
// number of candidates for the first pass, ceil(n_s ratio 1.15) + 64 with
// ratio the candidates per division seen last time: only a work estimate
// (more are drawn if it falls short; the selection does not depend on it),
// so FP32, as FP64 operations have long latencies here.
// (Not inlined: it runs once per launch, and two inlined copies would only
// add to the instruction fetches of a kernel that runs cold.)
static __device__ __noinline__ void plan_ns(double growth_rate, double rho_cell, long long mass_fix, double carry_in,
                                     double ratio_in, long long *ns_req, double *carry_out, double *kcf)
{
    const double mass = (double)mass_fix * kFixInv;
    const double xns = growth_rate * mass / rho_cell + carry_in;
    const double fl = floor(xns);
    *ns_req = (long long)fl;
    *carry_out = xns - fl;
    const float ratio = fmaxf((float)ratio_in, 1.0f);
    *kcf = (double)(ceilf((float)*ns_req * ratio * 1.15f) + 64.0f);
}

// The planner of one simulation, run by blocks blk = 0 .. G - 1 of PLAN_NT
// threads (all resident together when G > 1).
template <typename S, typename LT = Lat9>
__device__ __forceinline__ void plan_body(const SimDev &d, int init, int G, int blk)
{
    using R = arith_t<S>;
    DevScalars *sc = d.sc;
    // the state to observe is copy tn & 1, tn the step the selection is for:
    // the current step count for the initial state, else the next one
    const uint32_t tn = (uint32_t)sc->step + (init ? 0u : 1u);
    const int cur = (int)(tn & 1u);
    S *f = (S *)d.f[cur];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ long long s_ll[PLAN_WARPS];
    __shared__ int s_i[PLAN_WARPS], s_i2[PLAN_WARPS];
    __shared__ int s_dead;
    __shared__ unsigned long long s_kstop;
    __shared__ long long s_req;
    __shared__ double s_carry, s_kcf;
    // first-pass candidates of this block: key, and rank among the block's
    // accepted candidates (-1: rejected)
    __shared__ uint32_t s_key[PLAN_NT * PLAN_R];
    __shared__ int s_lr[PLAN_NT * PLAN_R];

    // the next update (launched as a programmatic dependent) may start its
    // prologue now; it waits for this grid's completion before reading
    grid_dependents_launch();
    // ---- the state left by the update that just ran (read before any block writes)
    const int y_r = sc->y_r, y_hi_old = sc->y_hi;
    const int maxmass = sc->maxmass_accum;
    const long long mass_acc = (long long)sc->mass_accum;
    const double carry_in = init ? sc->carry : sc->pend_carry;
    const double ratio_in = sc->acc_ratio;
    const bool grow = d.growth_mode != GROW_NONE;
    const long long wait_budget = sc->wait_budget > 0 ? sc->wait_budget : kWaitBudget;
    const int wait_extra = (sc->wait_test & WAIT_TEST_BARRIER) ? 1 : 0;
    // what block 0 commits at the end about the step that ran: its pending
    // statistics and the running totals, read before any block may write them
    __shared__ long long s_cm[11];
    __shared__ double s_cm_carry;
    if (blk == 0 && tid == 0) {
        s_cm[0] = sc->pend_req;
        s_cm[1] = sc->pend_acc;
        s_cm[2] = sc->pend_nev;
        s_cm[3] = sc->pend_cand;
        s_cm[4] = sc->ns_total;
        s_cm[5] = sc->div_total;
        s_cm[6] = sc->starved_steps;
        s_cm[7] = sc->node_updates;
        s_cm[8] = sc->step;
        s_cm[9] = sc->quiescent_fix;
        s_cm[10] = sc->pend_starved;
        s_cm_carry = sc->pend_carry;
    }
    if (tid == 0) {
        s_dead = 0;
        s_kstop = 0ull;
    }
    if (d.inject_in_update)
        for (int i = blk * PLAN_NT + tid; i < d.upd_ctas; i += G * PLAN_NT) d.bucket_cnt[i] = 0;
    // the previous selection's table entries emptied (before this selection
    // inserts, two grid barriers on)
    {
        const int nprev = sc->rec_n;
        for (int r = blk * PLAN_NT + tid; r < nprev; r += G * PLAN_NT) {
            const int slot = __ldcg(&d.hlist[r]);
            if (slot >= 0) d.htab[slot] = EMPTY_ENTRY;
        }
    }
    // n_s if no row is frozen now (almost always): the last block, which has
    // the least front to scan, works it out in FP64 while the others scan
    if (grow && blk == G - 1 && tid == 0) {
        long long req;
        double cy, kcf;
        plan_ns(d.growth_rate, d.rho_cell, mass_acc, carry_in, ratio_in, &req, &cy, &kcf);
        sc->spec_req = req;
        sc->spec_carry = cy;
        sc->spec_kcf = kcf;
    }

    // ---- A: front heights, per-block Eq. 6 sums
    int ytop = maxmass > y_r - 1 ? maxmass : y_r - 1;
    if (ytop > d.H - 1) ytop = d.H - 1;
    long long S1 = 0, S2 = 0;
    int top = 0, low = 0x7fffffff;
    for (int m = blk * PLAN_WARPS + warp; m < d.MW; m += G * PLAN_WARPS) {
        const int x = m * 32 + lane;
        unsigned pending = __ballot_sync(0xffffffffu, x < d.W);
        int h = 0;
        for (int yb = ytop; yb >= 0 && pending; yb -= 32) {
            // lane l loads row yb - l of the word; a 32 x 32 bit transpose
            // (five butterfly exchanges) gives lane c its column: bit l set
            // iff node (32 m + c, yb - l) is occupied
            const int y = yb - lane;
            unsigned col = y >= 0 ? d.mask[(long long)y * d.MW + m] : 0u;
#pragma unroll
            for (int j = 16; j > 0; j >>= 1) {
                const unsigned keep = j == 16 ? 0x0000FFFFu
                                    : j == 8  ? 0x00FF00FFu
                                    : j == 4  ? 0x0F0F0F0Fu
                                    : j == 2  ? 0x33333333u
                                              : 0x55555555u; // bits c with (c & j) == 0
                const unsigned other = __shfl_xor_sync(0xffffffffu, col, j);
                col = (lane & j) ? ((col & ~keep) | ((other & ~keep) >> j)) : ((col & keep) | ((other & keep) << j));
            }
            // the highest occupied row of a column not found above
            if (((pending >> lane) & 1u) && col != 0u) h = yb - (__ffs(col) - 1) + 1;
            pending &= ~__ballot_sync(0xffffffffu, col != 0u);
        }
        if (x < d.W) {
            d.heights[x] = h;
            S1 += h;
            S2 += (long long)h * h;
            top = max(top, h);
            low = min(low, h);
        }
    }
    {
        const long long a = plan_block_sum(S1, s_ll);
        const long long b2 = plan_block_sum(S2, s_ll);
        top = warp_max_i(top);
        low = warp_min_i(low);
        if (lane == 0) {
            s_i[warp] = top;
            s_i2[warp] = low;
        }
        __syncthreads();
        if (tid == 0) {
            int tp = 0, lw = 0x7fffffff;
            for (int i = 0; i < PLAN_WARPS; ++i) {
                tp = max(tp, s_i[i]);
                lw = min(lw, s_i2[i]);
            }
            d.pl_s1[blk] = a;
            d.pl_s2[blk] = b2;
            d.pl_top[blk] = tp;
            d.pl_low[blk] = lw;
        }
    }
    plan_grid_sync(sc, &s_dead, G, wait_budget, wait_extra);

    // ---- B: Eq. 6 sums, the rear wall, the active mass and the next plan
    // (every block computes the same values from the same partials)
    const bool advancing = d.wall_mode == 1 && !d.y_periodic;
    const bool need_s = blk == 0 || advancing;
    long long S1a = 0, S2a = 0;
    int topa = 0, lowa = 0x7fffffff;
    for (int i = tid; i < G; i += PLAN_NT) {
        if (need_s) {
            S1a += __ldcg(&d.pl_s1[i]);
            S2a += __ldcg(&d.pl_s2[i]);
        }
        topa = max(topa, __ldcg(&d.pl_top[i]));
        lowa = min(lowa, __ldcg(&d.pl_low[i]));
    }
    if (tid == 0 && grow) {
        s_req = __ldcg(&sc->spec_req);
        s_carry = __ldcg(&sc->spec_carry);
        s_kcf = __ldcg(&sc->spec_kcf);
    }
    if (need_s) { // uniform
        S1a = plan_block_sum(S1a, s_ll);
        S2a = plan_block_sum(S2a, s_ll);
    }
    topa = warp_max_i(topa);
    lowa = warp_min_i(lowa);
    if (lane == 0) {
        s_i[warp] = topa;
        s_i2[warp] = lowa;
    }
    __syncthreads();
    topa = 0;
    lowa = 0x7fffffff;
    for (int i = 0; i < PLAN_WARPS; ++i) {
        topa = max(topa, s_i[i]);
        lowa = min(lowa, s_i2[i]);
    }
    // the rear wall is kept behind the front at all times, the initial state
    // included: y_r <- max(y_r, floor(hbar - max(gap, 10 w))), Eq. 6 for w.
    // A float estimate first; the FP64 rule (as the oracle) only decides when
    // the wall can move
    int nyr = y_r;
    if (advancing) {
        const long long var = (long long)d.W * S2a - S1a * S1a;
        const float hf = (float)S1a / (float)d.W;
        const float wf = sqrtf((float)var) / (float)d.W;
        const float cf = hf - fmaxf((float)d.wall_min_gap, (float)d.wall_w_factor * wf);
        if (cf > (float)y_r + 0.9f) {
            const double hbar = (double)S1a / (double)d.W;
            const double wdt = sqrt((double)var) / (double)d.W;
            double gap = d.wall_min_gap;
            const double wg = d.wall_w_factor * wdt;
            if (wg > gap) gap = wg;
            double c = floor(hbar - gap);
            if (c > (double)(d.H - 1)) c = (double)(d.H - 1);
            const int cand = (int)c;
            if (cand > nyr) nyr = cand;
        }
    }
    // mass of the rows the wall freezes now
    long long frozen = 0;
    if (nyr > y_r) { // uniform across the grid
        const long long n = (long long)(nyr - y_r) * d.W;
        long long fm = 0;
        for (long long k = (long long)blk * PLAN_NT + tid; k < n; k += (long long)G * PLAN_NT) {
            const int y = y_r + (int)(k / d.W), x = (int)(k % d.W);
            const long long o = (long long)y * d.Wp + x;
            const Pop<S> pc(d);
            R r = pc.ld(f[o], 0);
#pragma unroll
            for (int i = 1; i < LT::Q; ++i) r = r + pc.ld(f[i * d.P + o], i);
            fm += fix24<R>(r);
        }
        fm = plan_block_sum(fm, s_ll);
        if (tid == 0) d.pl_mass[blk] = fm;
        plan_grid_sync(sc, &s_dead, G, wait_budget, wait_extra);
        long long a = 0;
        for (int i = tid; i < G; i += PLAN_NT) a += __ldcg(&d.pl_mass[i]);
        frozen = plan_block_sum(a, s_ll);
        if (tid == 0 && grow) {
            long long req;
            double cy, kcf;
            plan_ns(d.growth_rate, d.rho_cell, mass_acc - frozen, carry_in, ratio_in, &req, &cy, &kcf);
            s_req = req;
            s_carry = cy;
            s_kcf = kcf;
        }
    }
    __syncthreads();
    const long long mass_fix = mass_acc - frozen;
    // the window of the coming step (as block 0 commits it below): rows
    // [nyr, yhi_next) hold all the mass; the window never shrinks
    int yhi_next;
    if (d.y_periodic) {
        yhi_next = d.H;
    } else {
        yhi_next = maxmass + 2 < d.H ? maxmass + 2 : d.H;
        if (!init && y_hi_old > yhi_next) yhi_next = y_hi_old;
    }
    // proliferation plan (Sec. II): n_s sites, drawn from the active portion
    // restricted by the growth mode
    long long ns_req = 0, ns = 0, kc = 0;
    double carry_out = carry_in;
    int ylo = nyr, capacity = 0, nwin_zero = 0;
    unsigned long long nwin = 0ull;
    if (grow) {
        ns_req = s_req;
        carry_out = s_carry;
        ns = ns_req;
        int yhi_c = topa;
        if (d.growth_mode == GROW_EDGE) {
            const int e = lowa - d.edge_depth;
            if (e > ylo) ylo = e;
        } else if (d.growth_mode == GROW_BAND) {
            if (nyr + d.band_rows < yhi_c) yhi_c = nyr + d.band_rows;
        }
        nwin = yhi_c > ylo ? (unsigned long long)(yhi_c - ylo) * (unsigned long long)d.W : 0ull;
        // more than the planner holds, or a negative request (the exact
        // fixed-point mass overflowed: only a runaway lattice gets there):
        // no divisions this step, and the status says so
        if (ns > d.ns_max || ns < 0 || mass_fix < 0) {
            capacity = 1;
            ns = 0;
        }
        nwin_zero = (ns > 0 && nwin == 0) ? 1 : 0;
        if (nwin == 0) ns = 0;
        // candidates of the first pass: n_s times the ratio seen last step,
        // with a margin; more are drawn below if it falls short
        kc = (long long)s_kcf;
        const long long cap = 64 * ns + 1024;
        if (kc > cap) kc = cap;
        const long long kmax = (long long)G * PLAN_NT * PLAN_R;
        if (kc > kmax) kc = kmax;
        if (ns <= 0) kc = 0;
    }
    const size_t buf = (size_t)(tn & 1u) * (size_t)d.ns_max; // event list of step tn
    // counts of this selection start at zero (the selection below adds to
    // them after the next grid barrier)
    for (long long r = (long long)blk * PLAN_NT + tid; r < ns; r += (long long)G * PLAN_NT) d.ev_count[buf + r] = 0;

    // ---- C/D: candidates in draw order, the first n_s accepted, merged
    long long acc = 0; // accepted candidates so far (all blocks agree)
    if (ns > 0) {      // uniform
        const long long cap = 64 * ns + 1024;
        // first pass: block blk draws candidates [blk C, blk C + C); in round
        // i thread tid takes candidate blk C + i PLAN_NT + tid, so that the
        // gathers of a round are all in flight together
        const long long C = (kc + G - 1) / G;
        const int rounds = (int)((C + PLAN_NT - 1) / PLAN_NT); // <= PLAN_R (kc <= kmax)
        // (the round loops are not unrolled: this kernel runs with a cold
        // instruction cache, and every copy of the candidate code costs fetches)
        int tot_b = 0;
#pragma unroll 1
        for (int i = 0; i < rounds; ++i) {
            const long long j = (long long)i * PLAN_NT + tid;
            const long long k = (long long)blk * C + j;
            bool a = false;
            uint32_t key = 0u;
            if (j < C && k < kc) {
                const Candidate c = draw_candidate<LT>(d, k, tn, ylo, nwin);
                a = plan_accept<S, LT>(d, f, nyr, c);
                key = pack_key(c.x, c.y, c.pair);
            }
            int t_i;
            const int pre = plan_block_exscan(a ? 1 : 0, &t_i, s_i);
            s_key[j] = key;
            s_lr[j] = a ? tot_b + pre : -1;
            tot_b += t_i;
        }
        if (tid == 0) d.pl_cnt[blk] = tot_b;
        plan_grid_sync(sc, &s_dead, G, wait_budget, wait_extra);
        long long before = 0, total = 0;
        for (int i = tid; i < G; i += PLAN_NT) {
            const long long c = __ldcg(&d.pl_cnt[i]);
            total += c;
            before += i < blk ? c : 0;
        }
        before = plan_block_sum(before, s_ll);
        total = plan_block_sum(total, s_ll);
#pragma unroll 1
        for (int i = 0; i < rounds; ++i) {
            const int j = i * PLAN_NT + tid;
            const int lr = s_lr[j];
            if (lr >= 0) {
                const long long rank = before + lr;
                if (rank == ns - 1) s_kstop = (unsigned long long)(blk * C + j + 1);
                if (rank < ns) plan_select<R, LT>(d, s_key[j], (int)rank, buf, nyr);
            }
        }
        acc = total;
        // more draws, a grid-wide round at a time, while short of n_s: a
        // round is PLAN_R candidates per thread, thread tid of block blk
        // taking the PLAN_R consecutive ones from base + (blk PLAN_NT + tid)
        // PLAN_R, so that one block scan per round ranks them in draw order
        // (a member that accepts few candidates, whose growth starves, draws
        // up to the cap every step: fewer rounds, fewer barriers)
        long long base = kc;
        int round = 1;
        __syncthreads(); // (the first pass's entries of s_key, s_lr are read by other threads than the next writers)
        while (acc < ns && base < cap) { // uniform
            const long long k0 = base + ((long long)blk * PLAN_NT + tid) * PLAN_R;
            int mine = 0;
#pragma unroll 1
            for (int i = 0; i < PLAN_R; ++i) {
                const long long k = k0 + i;
                bool a = false;
                uint32_t key = 0u;
                if (k < cap) {
                    const Candidate c = draw_candidate<LT>(d, k, tn, ylo, nwin);
                    a = plan_accept<S, LT>(d, f, nyr, c);
                    key = pack_key(c.x, c.y, c.pair);
                }
                s_key[tid * PLAN_R + i] = key;
                s_lr[tid * PLAN_R + i] = a ? mine : -1;
                mine += a ? 1 : 0;
            }
            int tot_r;
            const int pr = plan_block_exscan(mine, &tot_r, s_i);
            int *cnt = d.pl_cnt + (round & 1) * kPlanMaxBlocks;
            if (tid == 0) cnt[blk] = tot_r;
            plan_grid_sync(sc, &s_dead, G, wait_budget, wait_extra);
            long long bf = 0, tt = 0;
            for (int i = tid; i < G; i += PLAN_NT) {
                const long long c = __ldcg(&cnt[i]);
                tt += c;
                bf += i < blk ? c : 0;
            }
            bf = plan_block_sum(bf, s_ll);
            tt = plan_block_sum(tt, s_ll);
#pragma unroll 1
            for (int i = 0; i < PLAN_R; ++i) {
                const int lr = s_lr[tid * PLAN_R + i];
                if (lr < 0) continue;
                const long long rank = acc + bf + pr + lr;
                if (rank == ns - 1) s_kstop = (unsigned long long)(k0 + i + 1);
                if (rank < ns) plan_select<R, LT>(d, s_key[tid * PLAN_R + i], (int)rank, buf, nyr);
            }
            acc += tt;
            base += (long long)G * PLAN_NT * PLAN_R;
            ++round;
        }
        __syncthreads();
        // the block that accepted the n_s-th candidate records how many were
        // drawn up to it, and the candidates per division for the next step
        if (tid == 0 && s_kstop) {
            sc->pend_cand = (long long)s_kstop;
            sc->acc_ratio = (double)((float)s_kstop / (float)ns); // a work estimate only
        }
    }
    // (no barrier: the commit below reads nothing another block writes after
    // the last one, and the table is emptied by the next launch)
    const int nsel = (int)(acc < ns ? acc : ns); // selected divisions (draw ranks)

    // ---- block 0: commit the step that ran, the observables, the new selection
    if (blk == 0 && tid == 0) {
        const long long p_req = s_cm[0], p_acc = s_cm[1], p_nev = s_cm[2], p_cand = s_cm[3];
        const long long ns_tot = s_cm[4], div_tot = s_cm[5], starved = s_cm[6], nupd = s_cm[7];
        const long long step = s_cm[8], qfix = s_cm[9];
        const int p_starved = (int)s_cm[10];
        const double p_carry = s_cm_carry;
        if (!init) {
            sc->ns_last = p_req;
            sc->ns_total = ns_tot + p_req;
            sc->carry = p_carry;
            sc->div_total = div_tot + p_acc;
            sc->events_last = p_acc;
            sc->n_events = p_nev;
            sc->cand_last = p_cand;
            if (p_starved) {
                sc->starved_steps = starved + 1;
                atomicOr(&sc->status, ST_STARVED);
            }
            sc->node_updates = nupd + (long long)d.W * (long long)(y_hi_old > y_r ? y_hi_old - y_r : 0);
            sc->step = step + 1;
        }
        sc->S1 = S1a;
        sc->S2 = S2a;
        sc->H_top = topa;
        sc->hmin = lowa;
        sc->mass_fix = mass_fix;
        sc->quiescent_fix = qfix + frozen;
        const int yhi = yhi_next;
        sc->y_copy = y_r;
        sc->y_r = nyr;
        sc->y_hi = yhi;
        if (maxmass >= d.H - 1) atomicOr(&sc->status, ST_FRONT_AT_TOP);
        if (capacity) atomicOr(&sc->status, ST_CAPACITY);
        sc->mass_accum = 0ull;
        sc->maxmass_accum = -1;
        // the selection for step tn, applied by the next update
        const long long cap = 64 * ns + 1024;
        sc->pend_req = ns_req;
        sc->pend_carry = carry_out;
        sc->pend_acc = nsel;
        sc->pend_nev = nsel;
        sc->pend_starved = (nwin_zero || (ns > 0 && acc < ns)) ? 1 : 0;
        // (with n_s reached, the accepting block wrote pend_cand and acc_ratio)
        if (!(ns > 0 && acc >= ns)) sc->pend_cand = nwin_zero ? 0 : (ns > 0 ? cap : 0);
        sc->plan_req = ns_req;
        sc->plan_ns = ns;
        sc->plan_kc = kc;
        sc->plan_ylo = ylo;
        sc->plan_nwin = nwin;
        sc->plan_carry = carry_out;
        sc->rec_n = nsel;
    }
    // the last block out restarts the barrier counter for the next launch (a
    // block counts itself out only after passing all its barriers, so no
    // block waits on the counter any more)
    if (G > 1) {
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            if (atomicAdd(&sc->plan_exit, 1u) == (unsigned)G - 1u) {
                sc->bar_ctr = 0ull;
                sc->plan_exit = 0u;
                __threadfence();
            }
        }
    }
}

// The planner of one simulation on a cooperative grid (launch_plan).
template <typename S, typename LT = Lat9>
__global__ void __launch_bounds__(PLAN_NT) k_plan(SimDev d, int init)
{
    plan_body<S, LT>(d, init, (int)gridDim.x, (int)blockIdx.x);
}

// The planners of a batch's slots in one cooperative launch of `cap` blocks
// (all resident at once), dealt on the device, every step, by the members'
// planner work: w = the candidates drawn for the latest selection (plan_work,
// copied by the injection launch before this one, so that it holds still
// while the planners run) + the lattice width (the front scans) + a fixed
// floor (the barriers and the commit). With tau = ceil(sum of w / (cap - 1)),
// a member with w >= tau is planned by G = floor(w / tau) blocks (at most
// kPlanMaxBlocks; the grid barrier on its own arrival counter, reset at the
// end of each launch, so the grid may change from step to step). The others
// (light) each get a block of their own when the heavy members' blocks and
// one per light member fit in the launch (a member's plan is mostly latency,
// so two in one block take twice as long); else they go, in slot order, into
// bins of about tau work, bin k holding the members whose prefix of light
// work lies in [k tau, (k + 1) tau), and a bin's block plans them one after
// another. The heavy members' blocks and the bins number at most
// sum w / tau + 1 <= cap. Every block computes the same deal from the same
// integers (counts and prefixes over the slots, in slot order).
constexpr long long kPlanWorkFloor = 4096;

__device__ __forceinline__ long long plan_slot_work(const SimDev *__restrict__ ds, int i)
{
    const DevScalars *sc = ds[i].sc;
    if (!sc) return -1; // an empty slot
    const long long c = sc->plan_work;
    return (c > 0 ? c : 0) + ds[i].W + kPlanWorkFloor;
}

template <typename S, typename LT = Lat9>
__global__ void __launch_bounds__(PLAN_NT, 2) k_plan_batch(const SimDev *__restrict__ ds, int nslots)
{
    __shared__ int s_hpre[kMaxBatchSlots + 1];       // heavy members' blocks, exclusive prefix
    __shared__ long long s_lpre[kMaxBatchSlots + 1]; // light members' work, exclusive prefix
    __shared__ long long s_red[PLAN_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cap = (int)gridDim.x;
    long long wsum = 0;
    for (int i = tid; i < nslots; i += PLAN_NT) {
        const long long w = plan_slot_work(ds, i);
        wsum += w > 0 ? w : 0;
    }
    wsum = plan_block_sum(wsum, s_red);
    if (wsum == 0) return; // (uniform: no members)
    const long long tau = (wsum + cap - 2) / (cap - 1);
    // one block per light member if that fits with the heavy members' blocks
    long long need = 0;
    for (int i = tid; i < nslots; i += PLAN_NT) {
        const long long w = plan_slot_work(ds, i);
        if (w >= tau) need += w / tau < kPlanMaxBlocks ? w / tau : kPlanMaxBlocks;
        else if (w >= 0) need += 1;
    }
    need = plan_block_sum(need, s_red);
    const bool own = need <= cap;           // (uniform)
    const long long bin = own ? 1 : tau;    // a bin's size in light-member units
    long long hrun = 0, lrun = 0;
    for (int base = 0; base < nslots; base += PLAN_NT) {
        const int i = base + tid;
        long long hg = 0, lw = 0;
        if (i < nslots) {
            const long long w = plan_slot_work(ds, i);
            if (w >= tau) hg = w / tau < kPlanMaxBlocks ? w / tau : kPlanMaxBlocks;
            else if (w >= 0) lw = own ? 1 : w;
        }
        // two exclusive block scans (64-bit: the work sums)
        long long ih = hg, il = lw;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long uh = __shfl_up_sync(0xffffffffu, ih, o);
            const long long ul = __shfl_up_sync(0xffffffffu, il, o);
            if (lane >= o) {
                ih += uh;
                il += ul;
            }
        }
        __shared__ long long s_wh[PLAN_WARPS], s_wl[PLAN_WARPS];
        if (lane == 31) {
            s_wh[warp] = ih;
            s_wl[warp] = il;
        }
        __syncthreads();
        long long bh = hrun + ih - hg, bl = lrun + il - lw, ch = 0, cl = 0;
        for (int k = 0; k < PLAN_WARPS; ++k) {
            if (k < warp) {
                bh += s_wh[k];
                bl += s_wl[k];
            }
            ch += s_wh[k];
            cl += s_wl[k];
        }
        if (i < nslots) {
            s_hpre[i] = (int)bh;
            s_lpre[i] = bl;
        }
        hrun += ch;
        lrun += cl;
        __syncthreads();
    }
    if (tid == 0) {
        s_hpre[nslots] = (int)hrun;
        s_lpre[nslots] = lrun;
    }
    __syncthreads();
    const int b = (int)blockIdx.x;
    if (b < (int)hrun) {
        // a heavy member's block: the last slot with s_hpre <= b
        int lo = 0, hi = nslots - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_hpre[mid] <= b) lo = mid; else hi = mid - 1;
        }
        const long long w = plan_slot_work(ds, lo);
        const int G = (int)(w / tau < kPlanMaxBlocks ? w / tau : kPlanMaxBlocks);
        plan_body<S, LT>(ds[lo], 0, G, b - s_hpre[lo]);
        return;
    }
    // bin k: the light members whose prefix (of work, or of members when
    // each has its own block) lies in [k bin, (k + 1) bin)
    const long long k = b - hrun, lo_w = k * bin, hi_w = lo_w + bin;
    if (lo_w >= lrun) return; // (uniform: no such bin)
    int lo = 0, hi = nslots; // the first slot with s_lpre >= lo_w
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_lpre[mid] < lo_w) lo = mid + 1; else hi = mid;
    }
    for (int i = lo; i < nslots && s_lpre[i] < hi_w; ++i) {
        const long long w = plan_slot_work(ds, i);
        if (w < 0 || w >= tau) continue; // empty, or heavy
        plan_body<S, LT>(ds[i], 0, 1, 0);
    }
}

// The batched planners' cooperative launch: `cap` blocks, at most the
// resident count.
template <typename S, typename LT = Lat9>
cudaError_t launch_plan_batch(const SimDev *ds, int nslots, int cap, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cap);
    cfg.blockDim = dim3(PLAN_NT);
    cfg.stream = s;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeCooperative;
    la[0].val.cooperative = 1;
    cfg.attrs = la;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_plan_batch<S, LT>, ds, nslots);
}

// App. A step 3 for the update kernels that read the populations from global
// memory: count * rho_cell/2 into the two pre-stream slots of each selected
// (node, pair) of step t, right before the update of step t. Distinct
// (node, pair) never share a slot (each slot streams into exactly one
// direction of one node).
// Division e (draw rank) of the step's selection.
template <typename S, typename LT = Lat9>
__device__ __forceinline__ void inject_division(const SimDev &d, S *f, int y_r, size_t buf, int e)
{
    using R = arith_t<S>;
    const Pop<S> pc(d);
    const int cnt = d.ev_count[buf + e];
    if (cnt == 0) return; // a repeat, counted at its first rank
    const uint32_t key = d.ev_key[buf + e];
    const int x = key_x(key), y = key_y(key), p = key_pair(key);
    const R add = (R)((double)cnt * d.half_cell);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = h == 0 ? LT::pa(p) : LT::pb(p);
        const long long o = LT::slot(d, y_r, x, y, q);
        // (the slot is in plane q or opp(q): one weight class)
        const S v = pc.st(pc.ld(f[o], q) + add, q);
        f[o] = v;
        // the ghost copy of an edge column (read by the TMA-staged update)
        const int xc = (int)((o % d.P) % d.Wp);
        if (xc == 0) f[o + d.W] = v;
        if (xc == d.W - 1) f[o - d.W] = v;
    }
}

template <typename S, typename LT = Lat9>
__device__ __forceinline__ void inject_body(const SimDev &d, int blk, int nblk)
{
    const uint32_t t = (uint32_t)d.sc->step;
    S *f = (S *)d.f[t & 1u];
    const int n = d.sc->rec_n, y_r = d.sc->y_r;
    const size_t buf = (size_t)(t & 1u) * (size_t)d.ns_max;
    for (int e = blk * (int)blockDim.x + (int)threadIdx.x; e < n; e += nblk * (int)blockDim.x)
        inject_division<S, LT>(d, f, y_r, buf, e);
}

template <typename S, typename LT = Lat9>
__global__ void k_inject(SimDev d)
{
    inject_body<S, LT>(d, (int)blockIdx.x, (int)gridDim.x);
}

// The injections of a batch's slots in one launch: every block forms, in
// shared memory, the exclusive prefix of the members' division counts (slot
// after slot; an empty slot, ds[m].sc == nullptr, has none) and the grid
// deals the batch's divisions, member after member, as one list. No table:
// members may come and go, and their planner capacities play no part.
constexpr int INJ_NT = 256;
template <typename S, typename LT = Lat9>
__global__ void __launch_bounds__(INJ_NT) k_inject_batch(const SimDev *__restrict__ ds, int nslots)
{
    __shared__ int s_pre[kMaxBatchSlots + 1];
    __shared__ int s_wsum[INJ_NT / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int run = 0; // divisions of the slots before this chunk
    for (int base = 0; base < nslots; base += INJ_NT) {
        const int m = base + tid;
        int n = 0;
        if (m < nslots) {
            const DevScalars *sc = ds[m].sc;
            if (sc) n = sc->rec_n;
        }
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        int before = run + incl - n, chunk = 0;
        for (int i = 0; i < INJ_NT / 32; ++i) {
            if (i < warp) before += s_wsum[i];
            chunk += s_wsum[i];
        }
        if (m < nslots) s_pre[m] = before;
        run += chunk;
        __syncthreads(); // (s_wsum is written again by the next chunk)
    }
    if (tid == 0) s_pre[nslots] = run;
    // the planners' work estimates, taken before they run (block 0)
    if (blockIdx.x == 0)
        for (int m = tid; m < nslots; m += INJ_NT) {
            DevScalars *sc = ds[m].sc;
            if (sc) sc->plan_work = sc->pend_cand;
        }
    __syncthreads();
    const int total = run;
    for (int g = (int)blockIdx.x * INJ_NT + tid; g < total; g += (int)gridDim.x * INJ_NT) {
        // the member of division g: the last m with s_pre[m] <= g
        int lo = 0, hi = nslots - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_pre[mid] <= g) lo = mid; else hi = mid - 1;
        }
        const SimDev &d = ds[lo];
        const uint32_t t = (uint32_t)d.sc->step;
        inject_division<S, LT>(d, (S *)d.f[t & 1u], d.sc->y_r, (size_t)(t & 1u) * (size_t)d.ns_max, g - s_pre[lo]);
    }
}

template <typename S, typename LT = Lat9>
cudaError_t launch_plan(const SimDev &d, int init, cudaStream_t s)
{
    // a cooperative launch: every block resident at once (the grid barriers
    // rely on it), or the launch fails
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)d.plan_grid);
    cfg.blockDim = dim3(PLAN_NT);
    cfg.stream = s;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeCooperative;
    la[0].val.cooperative = 1;
    cfg.attrs = la;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_plan<S, LT>, d, init);
}

// Resident blocks per SM of the planners: of k_plan (a simulation's own
// planner grid), or of k_plan_batch (`batch`: a batch's cooperative launch).
template <typename S, typename LT = Lat9>
int plan_blocks_per_sm(int batch)
{
    int n = 0;
    const cudaError_t e = batch ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_plan_batch<S, LT>, PLAN_NT, 0)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_plan<S, LT>, PLAN_NT, 0);
    return e == cudaSuccess ? n : 0;
}

} // namespace lbm
