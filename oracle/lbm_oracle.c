/*
 * Plain FP64 CPU oracle for the growing-tissue lattice Boltzmann method of
 * Killeen, Partridge, Bertrand & Lee, "Modeling growing confluent tissues using
 * a lattice Boltzmann method: interface stability and fluctuations"
 * (arXiv 2303.02210).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. The product path (the
 * CUDA library and its Python binding) never calls it, includes it or links it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes: App. A of the paper, one time step after another, over the
 * whole lattice (no active-window skipping), with two full population arrays
 * (current f and next f) plus the intermediate streamed distribution f*.
 * Everything is IEEE double; build with -ffp-contract=off so that no
 * multiply-add is fused and every operation rounds exactly where it is written.
 *
 * Lattice: D2Q9 by default (the D2Q9 analogue of Eq. 3 has coefficients 3,
 * 9/2, 3/2 and weights 4/9, 1/9, 1/36). Directions:
 *   0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)
 * or the paper's triangular D2Q7 (Sec. II): rows of nodes along x, the odd
 * rows shifted by half a spacing, rows sqrt(3)/2 apart; directions 0 rest and
 * q = 1..6 at angles (q - 1) pi / 3, i.e. 1:(1,0) 2:(1/2,s) 3:(-1/2,s)
 * 4:(-1,0) 5:(-1/2,-s) 6:(1/2,-s), s = sqrt(3)/2; Eq. 3 with 4, 8, 2
 * (c_s^2 = 1/4) and weights 1/2, 1/12. The neighbour of (x, y) along 2 is
 * (x + (y & 1), y + 1), along 3 (x - 1 + (y & 1), y + 1).
 * x is periodic (width W), y is the growth direction (height H). Node id
 * n = y*W + x. Population layout f[q][y][x], q-major.
 *
 * Per step t (App. A):
 *   1. streaming (Sec. II, two-step scheme): f*_i(x,y) = f_i(x-ex_i, y-ey_i);
 *      a source row outside [y_r, H) is a half-way bounce-back wall, so
 *      f*_i(x,y) = f_opp(i)(x,y) there (rear wall, Sec. III; top wall).
 *   2. rho* = sum_i f*_i, index order.
 *   3. proliferation (Sec. II, Eq. 5): n_s = floor(g*M/rho_cell + carry) sites,
 *      drawn with replacement from the active portion by a counter-based Philox
 *      stream; a candidate is accepted by the growth mode's rule on rho*;
 *      the first n_s accepted candidates in draw order are kept; each adds
 *      rho_cell/2 to the two populations of one opposite pair at its node.
 *   4. rho, u from f* (Eq. 1); u* = (1 - mu) u (Sec. II, below Eq. 3).
 *   5. redistribution (Eq. 2, Sec. II "two-step bounce-back"): if rho >= rho_c,
 *      f_i = f*_i - (f*_i - f^SS_i)/tau with f^SS from Eq. 3; else
 *      f_i = f*_opp(i).
 *   6. noise (Eq. 4) where rho >= rho_c.
 *   7. negative-population correction (App. A step 7).
 * Then: occupancy mask, front heights h(x), interface width w (Eq. 6), the
 * advancing rear wall (App. A, last paragraph), the active mass M.
 *
 * Parity is pinned by the tests in tests/test_oracle_*.py (Philox known-answer
 * vectors, exact mass conservation, closed-form momentum decay under friction,
 * shear-wave viscosity, ballistic streaming, two-step reversal of an isolated
 * sub-threshold node, growth ledger, selection statistics, Eq. 6 against a
 * library standard deviation).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NQ 9 /* the most directions of a lattice */

/* A lattice: q directions with vectors (ex, ey), opposites, weights, the
 * Eq. 3 coefficients f^SS_i = w_i rho (1 + c1 e.u + c2 (e.u)^2 - c3 u.u),
 * the opposite pairs a division may load (Sec. II: "two opposite lattice
 * vectors"; pair p touches pa[p] and pb[p]) and the bits of each Eq. 4
 * uniform (q fields of a 128-bit Philox block). */
typedef struct {
    int q, npairs, fbits;
    double ex[NQ], ey[NQ], w[NQ], c1, c2, c3;
    int opp[NQ], pa[4], pb[4];
} lattice;

#define HALF_SQRT3 0.8660254037844386 /* sqrt(3)/2, rounded to double */

static const lattice D2Q9 = {
    9, 4, 14,
    {0.0, 1.0, 0.0, -1.0, 0.0, 1.0, -1.0, -1.0, 1.0},
    {0.0, 0.0, 1.0, 0.0, -1.0, 1.0, 1.0, -1.0, -1.0},
    {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0},
    3.0, 4.5, 1.5,
    {0, 3, 4, 1, 2, 7, 8, 5, 6},
    {1, 2, 5, 6},
    {3, 4, 7, 8}};

static const lattice D2Q7 = {
    7, 3, 18,
    {0.0, 1.0, 0.5, -0.5, -1.0, -0.5, 0.5},
    {0.0, 0.0, HALF_SQRT3, HALF_SQRT3, 0.0, -HALF_SQRT3, -HALF_SQRT3},
    {0.5, 1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0},
    4.0, 8.0, 2.0,
    {0, 4, 5, 6, 1, 2, 3},
    {1, 2, 3},
    {4, 5, 6}};

enum { LATTICE_D2Q9 = 0, LATTICE_D2Q7 = 1 };

enum { GROW_NONE = 0, GROW_BULK = 1, GROW_DENSITY = 2, GROW_EDGE = 3, GROW_BAND = 4 };
enum { FRONT_FLAT = 0, FRONT_SINUSOIDAL = 1, FRONT_FULL = 2 };
enum { WALL_FIXED = 0, WALL_ADVANCE = 1 };
enum { NEGFIX_LITERAL = 0, NEGFIX_RESCALE = 1 };

/* Philox counter word 2 ("stream") for each use of random numbers. */
enum { STREAM_PROLIF = 1u, STREAM_INIT = 2u, STREAM_NOISE = 16u };

/* status bits */
enum { ORC_STATUS_FRONT_AT_TOP = 1, ORC_STATUS_GROWTH_STARVED = 2 };

typedef struct {
    double tau, mu, rho_c, rho_cell, sigma, rho0, growth_rate;
    double rho_init, rho_jitter, front_row, front_amp, wall_min_gap, wall_w_factor;
    uint64_t seed;
    int32_t width, height, growth_mode, edge_depth, band_rows, front_kind;
    int32_t front_kmin, front_kmax, wall_mode, negfix_mode, y_periodic;
    uint32_t sim_id;
    int32_t lattice; /* LATTICE_D2Q9 or LATTICE_D2Q7 */
} orc_params;

typedef struct {
    int64_t step, ns_last, ns_total, div_total, starved_steps, cand_last, events_last;
    int64_t mass_fix, quiescent_fix, S1, S2;
    double mass, quiescent_mass, carry, hbar, w, clip_mass;
    int32_t y_r, H_top, hmin, status;
} orc_stats;

typedef struct {
    orc_params p;
    const lattice *L;
    int W, H;
    size_t N;
    double *f, *fs, *fn; /* current, streamed (f*), next */
    uint8_t *mask;
    int32_t *h;
    /* proliferation bookkeeping of the last step */
    int64_t *ev_node;
    int32_t *ev_pair, *ev_count;
    int64_t ev_n, ev_cap;
    int64_t *acc_node; /* accepted candidates of this step, draw order */
    int32_t *acc_pair;
    int64_t acc_cap;
    orc_stats st;
} orc_sim;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11, "Parallel random numbers:
 * as easy as 1, 2, 3"): ten rounds of the 4x32 Philox S-box, key bumped by the
 * Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static void draw(const orc_sim *s, uint32_t a, uint32_t b, uint32_t stream, uint32_t out[4])
{
    uint32_t ctr[4] = {a, b, stream, s->p.sim_id};
    uint32_t key[2] = {(uint32_t)(s->p.seed & 0xFFFFFFFFu), (uint32_t)(s->p.seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Uniform on (0,1) from one 32-bit word: (v + 1/2) 2^-32, exact in double. */
static double u01(uint32_t v) { return ((double)v + 0.5) * 2.3283064365386963e-10; }

/* Node mass in the exact fixed-point unit 2^-24 (order-independent sums). */
static int64_t fix24(double r) { return llrint(r * 16777216.0); }

static double node_sum(const orc_sim *s, const double *f, size_t n)
{
    double r = f[n];
    for (int i = 1; i < s->L->q; ++i) r = r + f[(size_t)i * s->N + n];
    return r;
}

/* The node the population of direction i at (x, y) streams from (App. A
 * step 1: f*_i(x, y) = f_i(x - e_i, y - e_i) on D2Q9; on the triangular D2Q7,
 * the x offset of a step between rows depends on the row's parity), before
 * any wrap or wall. */
static void stream_source(const orc_sim *s, int i, int x, int y, int *xs, int *ys)
{
    if (s->p.lattice != LATTICE_D2Q7) {
        *xs = x - (int)s->L->ex[i];
        *ys = y - (int)s->L->ey[i];
        return;
    }
    const int par = y & 1;
    switch (i) {
    case 1: *xs = x - 1; *ys = y; break;
    case 2: *xs = x - 1 + par; *ys = y - 1; break; /* from the lower-left neighbour */
    case 3: *xs = x + par; *ys = y - 1; break;     /* from the lower-right neighbour */
    case 4: *xs = x + 1; *ys = y; break;
    case 5: *xs = x + par; *ys = y + 1; break;     /* from the upper-right neighbour */
    case 6: *xs = x - 1 + par; *ys = y + 1; break; /* from the upper-left neighbour */
    default: *xs = x; *ys = y; break;
    }
}

/* Momentum j = sum_i f_i e_i (Eq. 1), in a fixed order of operations. */
static void momentum(const orc_sim *s, const double *fs, double *jx, double *jy)
{
    if (s->p.lattice == LATTICE_D2Q7) {
        *jx = ((((fs[1] - fs[4]) + 0.5 * fs[2]) - 0.5 * fs[3]) - 0.5 * fs[5]) + 0.5 * fs[6];
        *jy = (((fs[2] + fs[3]) - fs[5]) - fs[6]) * HALF_SQRT3;
    } else {
        *jx = ((((fs[1] - fs[3]) + fs[5]) - fs[6]) - fs[7]) + fs[8];
        *jy = ((((fs[2] - fs[4]) + fs[5]) + fs[6]) - fs[7]) - fs[8];
    }
}

/* ------------------------------------------------------------------------ */
/* Observables: occupancy-derived front heights, Eq. 6 width, rear wall. */

static void compute_heights(orc_sim *s)
{
    const int W = s->W, H = s->H;
    int64_t S1 = 0, S2 = 0;
    int top = 0, low = H + 1;
    for (int x = 0; x < W; ++x) {
        int hx = 0;
        for (int y = H - 1; y >= 0; --y)
            if (s->mask[(size_t)y * W + x]) {
                hx = y + 1; /* h(x) = 1 + highest occupied row */
                break;
            }
        s->h[x] = hx;
        S1 += hx;
        S2 += (int64_t)hx * hx;
        if (hx > top) top = hx;
        if (hx < low) low = hx;
    }
    s->st.S1 = S1;
    s->st.S2 = S2;
    s->st.H_top = top;
    s->st.hmin = low;
    /* Eq. 6: w = sqrt(<h^2> - <h>^2), evaluated as sqrt(W S2 - S1^2) / W */
    s->st.hbar = (double)S1 / (double)W;
    s->st.w = sqrt((double)((int64_t)W * S2 - S1 * S1)) / (double)W;
}

static int64_t rows_mass_fix(const orc_sim *s, int y0, int y1)
{
    int64_t m = 0;
    for (int y = y0; y < y1; ++y)
        for (int x = 0; x < s->W; ++x) m += fix24(node_sum(s, s->f, (size_t)y * s->W + x));
    return m;
}

static void after_update(orc_sim *s)
{
    compute_heights(s);
    const int W = s->W, H = s->H;
    /* advancing rear wall: keep it at least max(gap, factor*w) behind hbar */
    if (s->p.wall_mode == WALL_ADVANCE && !s->p.y_periodic) {
        double gap = s->p.wall_min_gap;
        double wg = s->p.wall_w_factor * s->st.w;
        if (wg > gap) gap = wg;
        double c = floor(s->st.hbar - gap);
        if (c > (double)(H - 1)) c = (double)(H - 1);
        int cand = (int)c;
        if (cand > s->st.y_r) {
            s->st.quiescent_fix += rows_mass_fix(s, s->st.y_r, cand);
            s->st.y_r = cand;
        }
    }
    s->st.mass_fix = rows_mass_fix(s, s->st.y_r, H);
    s->st.mass = (double)s->st.mass_fix * 5.9604644775390625e-08;
    s->st.quiescent_mass = (double)s->st.quiescent_fix * 5.9604644775390625e-08;
    /* any mass in the top row: the front has reached the top wall */
    for (int x = 0; x < W; ++x)
        if (node_sum(s, s->f, (size_t)(H - 1) * W + x) != 0.0) {
            s->st.status |= ORC_STATUS_FRONT_AT_TOP;
            break;
        }
}

static void mask_from_state(orc_sim *s, int y0)
{
    for (int y = y0; y < s->H; ++y)
        for (int x = 0; x < s->W; ++x) {
            size_t n = (size_t)y * s->W + x;
            s->mask[n] = node_sum(s, s->f, n) >= s->p.rho_c;
        }
}

/* ------------------------------------------------------------------------ */
/* Initial condition (App. A, first paragraph): u = 0, f = f^SS(rho, 0) =
 * w_i rho; tissue below the initial front, empty above. */

static void init_state(orc_sim *s)
{
    const int W = s->W, H = s->H;
    const size_t N = s->N;
    int32_t *rows = (int32_t *)malloc(sizeof(int32_t) * W);
    if (s->p.front_kind == FRONT_FULL) {
        for (int x = 0; x < W; ++x) rows[x] = H;
    } else {
        double *h0 = (double *)malloc(sizeof(double) * W);
        if (s->p.front_kind == FRONT_FLAT) {
            for (int x = 0; x < W; ++x) {
                uint32_t r[4];
                draw(s, (uint32_t)x, 0u, STREAM_INIT, r);
                h0[x] = s->p.front_row + s->p.front_amp * (2.0 * u01(r[0]) - 1.0);
            }
        } else { /* sum of sinusoids with random phases, scaled to amplitude */
            const double two_pi = 6.283185307179586;
            double smax = 0.0;
            for (int x = 0; x < W; ++x) {
                double S = 0.0;
                for (int k = s->p.front_kmin; k <= s->p.front_kmax; ++k) {
                    uint32_t r[4];
                    draw(s, (uint32_t)k, 1u, STREAM_INIT, r);
                    double phi = two_pi * u01(r[0]);
                    S = S + sin(((two_pi * (double)k) * (double)x) / (double)W + phi);
                }
                h0[x] = S;
                if (fabs(S) > smax) smax = fabs(S);
            }
            for (int x = 0; x < W; ++x)
                h0[x] = smax > 0.0 ? s->p.front_row + s->p.front_amp * (h0[x] / smax) : s->p.front_row;
        }
        /* node (x, y) is tissue iff y < h0(x) */
        for (int x = 0; x < W; ++x) {
            double c = ceil(h0[x]);
            if (c < 0.0) c = 0.0;
            if (c > (double)H) c = (double)H;
            rows[x] = (int32_t)c;
        }
        free(h0);
    }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t n = (size_t)y * W + x;
            double rho = 0.0;
            if (y < rows[x]) {
                rho = s->p.rho_init;
                if (s->p.rho_jitter != 0.0) {
                    uint32_t r[4];
                    draw(s, (uint32_t)n, 2u, STREAM_INIT, r);
                    rho = s->p.rho_init * (1.0 + s->p.rho_jitter * (2.0 * u01(r[0]) - 1.0));
                }
            }
            for (int i = 0; i < s->L->q; ++i) s->f[(size_t)i * N + n] = s->L->w[i] * rho;
        }
    free(rows);
    mask_from_state(s, 0);
    after_update(s);
}

/* ------------------------------------------------------------------------ */
/* One time step, App. A steps 1-7. */

static int cmp_event(const void *a, const void *b)
{
    const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
    return (*x > *y) - (*x < *y);
}

static void one_step(orc_sim *s)
{
    const int W = s->W, H = s->H;
    const size_t N = s->N;
    const int yr = s->st.y_r;
    const uint32_t t = (uint32_t)s->st.step;
    const double rho_c = s->p.rho_c;

    /* ---- step 1: streaming into f* (rows of the active portion) ---- */
    const lattice *L = s->L;
    const int Q = L->q;
    for (int y = yr; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t n = (size_t)y * W + x;
            for (int i = 0; i < Q; ++i) {
                int xs, ys;
                stream_source(s, i, x, y, &xs, &ys);
                xs = (xs + W) % W;
                double v;
                if (s->p.y_periodic) {
                    ys = (ys + H) % H;
                    v = s->f[(size_t)i * N + (size_t)ys * W + xs];
                } else if (ys < yr || ys >= H) {
                    v = s->f[(size_t)L->opp[i] * N + n]; /* half-way bounce-back */
                } else {
                    v = s->f[(size_t)i * N + (size_t)ys * W + xs];
                }
                s->fs[(size_t)i * N + n] = v;
            }
        }

    /* ---- step 3: proliferation (acceptance uses rho* of step 2) ---- */
    int64_t ns = 0;
    s->ev_n = 0;
    s->st.cand_last = 0;
    if (s->p.growth_mode != GROW_NONE) {
        double x_ns = s->p.growth_rate * s->st.mass / s->p.rho_cell + s->st.carry;
        double fl = floor(x_ns);
        ns = (int64_t)fl;
        s->st.carry = x_ns - fl;
        /* candidate rows: the active portion, restricted per growth mode */
        int y_lo = yr, y_hi = s->st.H_top;
        if (s->p.growth_mode == GROW_EDGE) {
            int e = s->st.hmin - s->p.edge_depth;
            if (e > y_lo) y_lo = e;
        } else if (s->p.growth_mode == GROW_BAND) {
            if (yr + s->p.band_rows < y_hi) y_hi = yr + s->p.band_rows;
        }
        int64_t nwin = (y_hi > y_lo) ? (int64_t)(y_hi - y_lo) * W : 0;
        int64_t accepted = 0, k = 0;
        if (ns > 0 && nwin > 0) {
            int64_t cap = 64 * ns + 1024;
            if (s->acc_cap < ns) {
                s->acc_cap = ns;
                s->acc_node = (int64_t *)realloc(s->acc_node, sizeof(int64_t) * ns);
                s->acc_pair = (int32_t *)realloc(s->acc_pair, sizeof(int32_t) * ns);
            }
            for (k = 0; k < cap && accepted < ns; ++k) {
                uint32_t r[4];
                draw(s, (uint32_t)k, t, STREAM_PROLIF, r);
                int64_t idx = (int64_t)(((uint64_t)r[0] * (uint64_t)nwin) >> 32);
                int64_t node = (int64_t)y_lo * W + idx;
                int y = (int)(node / W), x = (int)(node % W);
                /* a pair uniform over the lattice's opposite pairs */
                int pair = L->npairs == 4 ? (int)(r[1] >> 30) : (int)(((uint64_t)r[1] * (uint64_t)L->npairs) >> 32);
                double rs = node_sum(s, s->fs, (size_t)node); /* rho* */
                int ok = 0;
                switch (s->p.growth_mode) {
                case GROW_BULK: ok = rs >= rho_c; break;
                case GROW_BAND: ok = rs >= rho_c; break;
                case GROW_EDGE: ok = rs >= rho_c && (s->h[x] - y) <= s->p.edge_depth; break;
                case GROW_DENSITY: /* Eq. 5 */
                    ok = rs > rho_c && u01(r[2]) < 1.0 - rs / s->p.rho0;
                    break;
                }
                if (ok) {
                    s->acc_node[accepted] = node;
                    s->acc_pair[accepted] = pair;
                    ++accepted;
                }
            }
        }
        s->st.cand_last = k;
        if (accepted < ns) {
            s->st.starved_steps += 1;
            s->st.status |= ORC_STATUS_GROWTH_STARVED;
        }
        /* sites drawn more than once add their count at once */
        int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (accepted > 0 ? accepted : 1));
        for (int64_t a = 0; a < accepted; ++a) key[a] = s->acc_node[a] * 4 + s->acc_pair[a];
        qsort(key, (size_t)accepted, sizeof(int64_t), cmp_event);
        if (s->ev_cap < accepted) {
            s->ev_cap = accepted;
            s->ev_node = (int64_t *)realloc(s->ev_node, sizeof(int64_t) * accepted);
            s->ev_pair = (int32_t *)realloc(s->ev_pair, sizeof(int32_t) * accepted);
            s->ev_count = (int32_t *)realloc(s->ev_count, sizeof(int32_t) * accepted);
        }
        const double half = s->p.rho_cell * 0.5;
        for (int64_t a = 0; a < accepted;) {
            int64_t b = a;
            while (b < accepted && key[b] == key[a]) ++b;
            int64_t node = key[a] / 4;
            int pair = (int)(key[a] % 4);
            int32_t cnt = (int32_t)(b - a);
            double add = (double)cnt * half;
            s->fs[(size_t)L->pa[pair] * N + (size_t)node] += add;
            s->fs[(size_t)L->pb[pair] * N + (size_t)node] += add;
            s->ev_node[s->ev_n] = node;
            s->ev_pair[s->ev_n] = pair;
            s->ev_count[s->ev_n] = cnt;
            s->ev_n += 1;
            a = b;
        }
        free(key);
        s->st.ns_last = ns;
        s->st.ns_total += ns;
        s->st.div_total += accepted;
        s->st.events_last = accepted;
    } else {
        s->st.ns_last = 0;
        s->st.events_last = 0;
    }

    /* ---- steps 4-7 per node ---- */
    const double omega = 1.0 / s->p.tau;
    const double cmu = 1.0 - s->p.mu;
    const double two_sigma = 2.0 * s->p.sigma;
    for (int y = yr; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t n = (size_t)y * W + x;
            double fs[NQ], fo[NQ];
            for (int i = 0; i < Q; ++i) fs[i] = s->fs[(size_t)i * N + n];
            /* step 4: moments of f* after proliferation (Eq. 1) */
            double rho = fs[0];
            for (int i = 1; i < Q; ++i) rho = rho + fs[i];
            int occ = rho >= rho_c;
            s->mask[n] = (uint8_t)occ;
            if (!occ) {
                /* step 5, rho < rho_c: reverse directions (two-step bounce-back) */
                for (int i = 0; i < Q; ++i) fo[i] = fs[L->opp[i]];
            } else {
                double jx, jy;
                momentum(s, fs, &jx, &jy);
                double ux = jx / rho, uy = jy / rho;
                double usx = cmu * ux, usy = cmu * uy; /* u* = (1 - mu) u */
                double uu = usx * usx + usy * usy;
                /* step 5, rho >= rho_c: BGK relaxation towards f^SS (Eqs. 2-3) */
                for (int i = 0; i < Q; ++i) {
                    double eu = L->ex[i] * usx + L->ey[i] * usy;
                    double t1 = 1.0 + L->c1 * eu;
                    t1 = t1 + L->c2 * (eu * eu);
                    t1 = t1 - L->c3 * uu;
                    double fss = (L->w[i] * rho) * t1;
                    fo[i] = fs[i] - omega * (fs[i] - fss);
                }
                /* step 6: mass-conserving noise (Eq. 4). Q uniforms u_i on (0,1)
                 * with b random bits each (D2Q9: 9 of 14 bits, D2Q7: 7 of 18),
                 * from one Philox block: its four words read as the 128-bit
                 * integer w0 + 2^32 w1 + 2^64 w2 + 2^96 w3, whose bits b i ..
                 * b i + b - 1 are m_i; u_i = (m_i + 1/2) 2^-b.
                 * eta~_i = sigma (2 u_i - 1), so eta_i = eta~_i - mean(eta~)
                 * = 2 sigma (u_i - mean(u)). */
                if (s->p.sigma != 0.0) {
                    uint32_t w[4];
                    draw(s, (uint32_t)n, t, STREAM_NOISE, w);
                    uint32_t m[NQ];
                    for (int i = 0; i < Q; ++i) {
                        const int bit = L->fbits * i, j = bit / 32, o = bit % 32;
                        uint64_t two = (uint64_t)w[j];
                        if (j + 1 < 4) two |= (uint64_t)w[j + 1] << 32;
                        m[i] = (uint32_t)(two >> o) & ((1u << L->fbits) - 1u);
                    }
                    double u[NQ];
                    for (int i = 0; i < Q; ++i) u[i] = ((double)m[i] + 0.5) * ldexp(1.0, -L->fbits);
                    double S = u[0];
                    for (int i = 1; i < Q; ++i) S = S + u[i];
                    const double ubar = S / (double)Q;
                    for (int i = 0; i < Q; ++i) fo[i] = fo[i] + two_sigma * (u[i] - ubar);
                }
                /* step 7: correct negative populations */
                if (s->p.negfix_mode == NEGFIX_LITERAL) {
                    if (fo[0] < 0.0) {
                        double r0 = fo[0];
                        for (int i = 1; i < Q; ++i) r0 = r0 + fo[i];
                        fo[0] = 0.0;
                        double sm = fo[0];
                        for (int i = 1; i < Q; ++i) sm = sm + fo[i];
                        for (int i = 0; i < Q; ++i) fo[i] = (r0 * fo[i]) / sm;
                    }
                    for (int i = 1; i < Q; ++i)
                        if (fo[i] < 0.0) {
                            double a = -fo[i];
                            fo[L->opp[i]] = fo[L->opp[i]] + a;
                            fo[i] = 0.0;
                            s->st.clip_mass += 2.0 * a;
                        }
                } else {
                    int neg = 0;
                    for (int i = 0; i < Q; ++i) neg |= fo[i] < 0.0;
                    if (neg) {
                        double r0 = fo[0];
                        for (int i = 1; i < Q; ++i) r0 = r0 + fo[i];
                        for (int i = 0; i < Q; ++i)
                            if (fo[i] < 0.0) fo[i] = 0.0;
                        double sm = fo[0];
                        for (int i = 1; i < Q; ++i) sm = sm + fo[i];
                        for (int i = 0; i < Q; ++i) fo[i] = (r0 * fo[i]) / sm;
                    }
                }
            }
            for (int i = 0; i < Q; ++i) s->fn[(size_t)i * N + n] = fo[i];
        }
    /* rows behind the rear wall are quiescent: unchanged */
    for (int i = 0; i < Q; ++i)
        if (yr > 0) memcpy(s->fn + (size_t)i * N, s->f + (size_t)i * N, sizeof(double) * (size_t)yr * W);
    double *tmp = s->f;
    s->f = s->fn;
    s->fn = tmp;
    s->st.step += 1;
    after_update(s);
}

/* ------------------------------------------------------------------------ */
/* C interface used by the Python wrapper (oracle/oracle.py). */

void *orc_create(const orc_params *p)
{
    if (p->width < 1 || p->height < 3 || (int64_t)p->width * p->height > (1 << 30)) return NULL;
    if (p->width > 32768 || p->height > 32768) return NULL;
    if (!(p->tau > 0.5) || !(p->rho_cell > 0.0) || !(p->rho_c >= 0.0)) return NULL;
    if (p->lattice != LATTICE_D2Q9 && p->lattice != LATTICE_D2Q7) return NULL;
    /* a y-periodic triangular lattice needs an even number of rows */
    if (p->lattice == LATTICE_D2Q7 && p->y_periodic && (p->height & 1)) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->p = *p;
    s->L = p->lattice == LATTICE_D2Q7 ? &D2Q7 : &D2Q9;
    s->W = p->width;
    s->H = p->height;
    s->N = (size_t)s->W * s->H;
    s->f = (double *)calloc((size_t)s->L->q * s->N, sizeof(double));
    s->fs = (double *)calloc((size_t)s->L->q * s->N, sizeof(double));
    s->fn = (double *)calloc((size_t)s->L->q * s->N, sizeof(double));
    s->mask = (uint8_t *)calloc(s->N, 1);
    s->h = (int32_t *)calloc(s->W, sizeof(int32_t));
    if (!s->f || !s->fs || !s->fn || !s->mask || !s->h) {
        free(s->f); free(s->fs); free(s->fn); free(s->mask); free(s->h); free(s);
        return NULL;
    }
    init_state(s);
    return s;
}

void orc_destroy(void *h)
{
    orc_sim *s = (orc_sim *)h;
    if (!s) return;
    free(s->f); free(s->fs); free(s->fn); free(s->mask); free(s->h);
    free(s->ev_node); free(s->ev_pair); free(s->ev_count);
    free(s->acc_node); free(s->acc_pair);
    free(s);
}

void orc_step(void *h, int64_t n)
{
    orc_sim *s = (orc_sim *)h;
    for (int64_t k = 0; k < n; ++k) one_step(s);
}

void orc_get_pops(void *h, double *out)
{
    orc_sim *s = (orc_sim *)h;
    memcpy(out, s->f, sizeof(double) * (size_t)s->L->q * s->N);
}

/* Replace the populations (e.g. a test's own initial state); the occupancy
 * mask of the active rows and the observables are recomputed from them. */
void orc_set_pops(void *h, const double *in)
{
    orc_sim *s = (orc_sim *)h;
    memcpy(s->f, in, sizeof(double) * (size_t)s->L->q * s->N);
    mask_from_state(s, s->st.y_r);
    s->st.status = 0;
    after_update(s);
}

void orc_get_mask(void *h, uint8_t *out)
{
    orc_sim *s = (orc_sim *)h;
    memcpy(out, s->mask, s->N);
}

void orc_get_heights(void *h, int32_t *out)
{
    orc_sim *s = (orc_sim *)h;
    memcpy(out, s->h, sizeof(int32_t) * s->W);
}

void orc_get_stats(void *h, orc_stats *out) { *out = ((orc_sim *)h)->st; }

/* rho and u = j/rho of the current populations (u = 0 where rho = 0). */
void orc_fields(void *h, double *rho, double *ux, double *uy)
{
    orc_sim *s = (orc_sim *)h;
    for (size_t n = 0; n < s->N; ++n) {
        double fs[NQ];
        for (int i = 0; i < s->L->q; ++i) fs[i] = s->f[(size_t)i * s->N + n];
        double r = fs[0];
        for (int i = 1; i < s->L->q; ++i) r = r + fs[i];
        double jx, jy;
        momentum(s, fs, &jx, &jy);
        rho[n] = r;
        ux[n] = r != 0.0 ? jx / r : 0.0;
        uy[n] = r != 0.0 ? jy / r : 0.0;
    }
}

/* Proliferation events of the last step, sorted by (node, pair). */
int64_t orc_last_events(void *h, int64_t *node, int32_t *pair, int32_t *count, int64_t cap)
{
    orc_sim *s = (orc_sim *)h;
    int64_t n = s->ev_n < cap ? s->ev_n : cap;
    for (int64_t a = 0; a < n; ++a) {
        node[a] = s->ev_node[a];
        pair[a] = s->ev_pair[a];
        count[a] = s->ev_count[a];
    }
    return s->ev_n;
}

int32_t orc_sizeof_params(void) { return (int32_t)sizeof(orc_params); }
int32_t orc_directions(void *h) { return (int32_t)((orc_sim *)h)->L->q; }
int32_t orc_sizeof_stats(void) { return (int32_t)sizeof(orc_stats); }
