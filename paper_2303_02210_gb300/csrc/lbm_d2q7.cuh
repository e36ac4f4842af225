// The paper's triangular D2Q7 lattice (Sec. II; Eq. 3 with coefficients 4, 8,
// 2 and weights 1/2, 1/12, c_s^2 = 1/4): the kernels whose arithmetic or
// streaming differ from D2Q9, in FP32 or FP64 storage (the planner and the
// injection are the D2Q9 ones on the Lat7 traits), and the division records
// of the TMA-staged D2Q7 update (lbm_update7_tma.cuh). Rows of nodes along x, odd
// rows shifted by half a spacing, rows sqrt(3)/2 apart; directions 0 rest and
// 1:(1,0) 2:(1/2,s) 3:(-1/2,s) 4:(-1,0) 5:(-1/2,-s) 6:(1/2,-s), s = sqrt(3)/2,
// opposites q <-> q + 3. Population layout f[q][y][x] with seven planes.
//
// The FP64 forms follow the CPU oracle operation by operation (bit-exact); the
// FP32 forms regroup as the D2Q9 fast path does (one reciprocal for u, f_0 from
// mass conservation, the noise uniforms from mantissa bits).
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

constexpr int NQ7 = 7;
constexpr double HALF_SQRT3 = 0.8660254037844386; // sqrt(3)/2 rounded to double

template <typename R>
__host__ __device__ constexpr R ex7(int q)
{
    return q == 1 ? R(1) : (q == 4 ? R(-1) : (q == 2 || q == 6 ? R(0.5) : (q == 3 || q == 5 ? R(-0.5) : R(0))));
}
template <typename R>
__host__ __device__ constexpr R ey7(int q)
{
    return q == 2 || q == 3 ? R(HALF_SQRT3) : (q == 5 || q == 6 ? R(-HALF_SQRT3) : R(0));
}
template <typename R>
__host__ __device__ constexpr R w7(int q)
{
    return q == 0 ? R(0.5) : R(1) / R(12);
}

// Initial state (App. A): f_i = w_i rho below the front, zero above, in both
// copies; the ghost columns x = -1 and x = W as for D2Q9.
template <typename S>
__global__ void k_fill7(SimDev d)
{
    S *f0 = (S *)d.f[0];
    S *f1 = (S *)d.f[1];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d.sc->maxmass_accum = -1;
        d.sc->low_acc = 0x7fffffff;
    }
    const long long total = (long long)d.H * d.Wp;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(idx / d.Wp), xs = (int)(idx % d.Wp) - kXO;
        const int x = xs == -1 ? d.W - 1 : (xs == d.W ? 0 : xs);
        double rho = 0.0;
        if (x >= 0 && x < d.W && y < d.rows0[x]) {
            rho = d.rho_init;
            if (d.rho_jitter != 0.0) {
                const u32x4 r = philox4x32_10(u32x4{(uint32_t)(y * d.W + x), 2u, STREAM_INIT, d.sim}, d.pk);
                rho = d.rho_init * (1.0 + d.rho_jitter * (2.0 * u01(r.x) - 1.0));
            }
        }
        const long long o = (long long)y * d.Wp + xs;
#pragma unroll
        for (int i = 0; i < NQ7; ++i) {
            const S v = (S)(w7<double>(i) * rho);
            f0[i * d.P + o] = v;
            f1[i * d.P + o] = v;
        }
    }
}

// Ghost columns of the seven planes of both copies.
template <typename S>
__global__ void k_ghosts7(SimDev d)
{
    const long long total = 2LL * NQ7 * d.H;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < 2 * total;
         k += (long long)gridDim.x * blockDim.x) {
        S *f = (S *)d.f[k >= total ? 1 : 0];
        const long long r = k >= total ? k - total : k;
        const int side = (int)(r & 1);
        const long long row = r >> 1; // plane * H + y
        S *base = f + (row / d.H) * d.P + (row % d.H) * d.Wp;
        if (side == 0)
            base[-1] = base[d.W - 1];
        else
            base[d.W] = base[0];
    }
}

// Occupancy mask, exact mass and highest mass row of rows [y_r, H) of copy cur.
template <typename S>
__global__ void k_scan7(SimDev d, int cur)
{
    using R = S;
    const S *f = (const S *)d.f[cur];
    const int y_r = d.sc->y_r;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long words = (long long)(d.H - y_r) * d.MW;
    long long mass = 0;
    int maxrow = -1;
    for (long long wi = (((long long)blockIdx.x * blockDim.x) + threadIdx.x) >> 5; wi < words; wi += nwarps) {
        const int y = y_r + (int)(wi / d.MW);
        const int m = (int)(wi % d.MW);
        const int x = m * 32 + lane;
        const bool ok = x < d.W;
        R rho = R(0);
        bool any = false;
        if (ok) {
            const long long n = (long long)y * d.Wp + x;
            rho = f[n];
            any = rho != R(0);
#pragma unroll
            for (int i = 1; i < NQ7; ++i) {
                const R v = f[i * d.P + n];
                rho = rho + v;
                any |= v != R(0);
            }
        }
        const unsigned b = __ballot_sync(0xffffffffu, ok && rho >= rho_c_of<R>(d));
        if (lane == 0) d.mask[(long long)y * d.MW + m] = b;
        if (ok) mass += fix24<R>(rho);
        if (any) maxrow = y;
    }
    mass = warp_sum_ll(mass);
    maxrow = warp_max_i(maxrow);
    if (lane == 0) {
        atomicAdd(&d.sc->mass_accum, (unsigned long long)mass);
        atomicMax(&d.sc->maxmass_accum, maxrow);
    }
}

// Momentum j = sum_i f_i e_i in the oracle's order of operations.
template <typename R>
__device__ __forceinline__ void momentum7(const R *g, R &jx, R &jy)
{
    jx = ((((g[1] - g[4]) + R(0.5) * g[2]) - R(0.5) * g[3]) - R(0.5) * g[5]) + R(0.5) * g[6];
    jy = (((g[2] + g[3]) - g[5]) - g[6]) * R(HALF_SQRT3);
}

// rho and u of copy cur into device arrays of W*H doubles (Eq. 1).
template <typename S>
__global__ void k_fields7(SimDev d, int cur, double *rho, double *ux, double *uy)
{
    const S *f = (const S *)d.f[cur];
    const long long total = (long long)d.W * d.H;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / d.W), x = (int)(k % d.W);
        const long long o = (long long)y * d.Wp + x;
        double g[NQ7];
#pragma unroll
        for (int i = 0; i < NQ7; ++i) g[i] = (double)f[i * d.P + o];
        double r = g[0];
#pragma unroll
        for (int i = 1; i < NQ7; ++i) r = r + g[i];
        double jx, jy;
        momentum7<double>(g, jx, jy);
        rho[k] = r;
        ux[k] = r != 0.0 ? jx / r : 0.0;
        uy[k] = r != 0.0 ? jy / r : 0.0;
    }
}

// ===========================================================================
// Per-node collision (Eqs. 2-4 and App. A step 7) on seven directions.

// The seven 18-bit fields of a Philox block read as one 128-bit integer
// w.x + 2^32 w.y + 2^64 w.z + 2^96 w.w: field i is bits 18 i .. 18 i + 17.
__device__ __forceinline__ void noise_fields7(const u32x4 &w, uint32_t m[NQ7])
{
    m[0] = w.x;
    m[1] = __funnelshift_r(w.x, w.y, 18);
    m[2] = w.y >> 4;
    m[3] = __funnelshift_r(w.y, w.z, 22);
    m[4] = w.z >> 8;
    m[5] = __funnelshift_r(w.z, w.w, 26);
    m[6] = w.w >> 12;
#pragma unroll
    for (int i = 0; i < NQ7; ++i) m[i] &= 0x3FFFFu;
}

// Eqs. 2-3 (and Eq. 4: eta added, or nothing if eta is null) for an occupied
// node; FP64 in the oracle's order, FP32 regrouped.
template <typename R>
__device__ __forceinline__ void collide7(const R *g, R rho, R *fo, const Consts<R> &c, const R *eta)
{
    R jx, jy;
    momentum7<R>(g, jx, jy);
    if constexpr (sizeof(R) == 8) {
        const R ux = jx / rho, uy = jy / rho;
        const R usx = c.cmu * ux, usy = c.cmu * uy; // u* = (1 - mu) u
        const R uu = usx * usx + usy * usy;
#pragma unroll
        for (int i = 0; i < NQ7; ++i) {
            const R eu = ex7<R>(i) * usx + ey7<R>(i) * usy;
            R t1 = R(1) + R(4) * eu;
            t1 = t1 + R(8) * (eu * eu);
            t1 = t1 - R(2) * uu;
            const R fss = (w7<R>(i) * rho) * t1;    // Eq. 3, D2Q7
            fo[i] = g[i] - c.omega * (g[i] - fss); // Eq. 2
        }
        if (eta) {
#pragma unroll
            for (int i = 0; i < NQ7; ++i) fo[i] = fo[i] + eta[i]; // Eq. 4
        }
    } else {
        float rr;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rr) : "f"(rho));
        const float k = c.cmu * rr;
        const float usx = jx * k, usy = jy * k;
        const float A = fmaf(-2.0f, fmaf(usx, usx, usy * usy), 1.0f);
        const float r1 = (1.0f / 12.0f) * rho;
        // opposite pairs share 1 + 8 (e.u)^2 - 2 u.u and differ in the sign of 4 e.u
#pragma unroll
        for (int p = 1; p <= 3; ++p) {
            const float e = ex7<float>(p) * usx + ey7<float>(p) * usy;
            const float base = fmaf(8.0f * e, e, A);
            const float fa = r1 * fmaf(4.0f, e, base), fb = r1 * fmaf(-4.0f, e, base);
            fo[p] = fmaf(c.om1, g[p], fmaf(c.omega, fa, eta ? eta[p] : 0.0f));
            fo[p + 3] = fmaf(c.om1, g[p + 3], fmaf(c.omega, fb, eta ? eta[p + 3] : 0.0f));
        }
        // f_0 = rho - sum_{i>0} f_i: the relaxation and the noise conserve the
        // node's mass exactly, and this keeps rounding from drifting it
        fo[0] = rho - (((fo[1] + fo[2]) + (fo[3] + fo[4])) + (fo[5] + fo[6]));
    }
}

// Eq. 4: eta_i = 2 sigma (u_i - mean u), u_i = (m_i + 1/2) 2^-18 with m_i the
// 18-bit fields of the node's Philox block (n, t, 16, sim).
template <typename R>
__device__ __forceinline__ void noise_eta7(R *eta, const u32x4 &w, const Consts<R> &c)
{
    uint32_t m[NQ7];
    noise_fields7(w, m);
    if constexpr (sizeof(R) == 8) {
        double u[NQ7];
#pragma unroll
        for (int i = 0; i < NQ7; ++i) u[i] = ((double)m[i] + 0.5) * 3.814697265625e-06;
        double S = u[0];
#pragma unroll
        for (int i = 1; i < NQ7; ++i) S = S + u[i];
        const double ubar = S / 7.0;
#pragma unroll
        for (int i = 0; i < NQ7; ++i) eta[i] = c.two_sigma * (u[i] - ubar);
    } else {
        // 1 + m 2^-18 exactly; the constant offset cancels in u_i - mean u
        float v[NQ7];
#pragma unroll
        for (int i = 0; i < NQ7; ++i) v[i] = __uint_as_float(0x3F800000u | (m[i] << 5));
        const float S = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + v[6]);
        const float nb = -c.two_sigma * (S * (1.0f / 7.0f));
        eta[0] = 0.0f; // f_0 follows from mass conservation
#pragma unroll
        for (int i = 1; i < NQ7; ++i) eta[i] = fmaf(c.two_sigma, v[i], nb);
    }
}

// App. A step 7 on seven directions (as fix_negative for D2Q9). Returns the
// mass the fix added.
template <typename R>
__device__ __forceinline__ R fix_negative7(R *fo, int mode)
{
    R added = R(0);
    R mn = fo[0];
#pragma unroll
    for (int i = 1; i < NQ7; ++i) mn = mn < fo[i] ? mn : fo[i];
    if (!(mn < R(0))) return added;
    if (mode == 0) { // LITERAL (else RESCALE)
        if (fo[0] < R(0)) {
            R r0 = fo[0];
#pragma unroll
            for (int i = 1; i < NQ7; ++i) r0 = r0 + fo[i];
            fo[0] = R(0);
            R sm = fo[0];
#pragma unroll
            for (int i = 1; i < NQ7; ++i) sm = sm + fo[i];
#pragma unroll
            for (int i = 0; i < NQ7; ++i) fo[i] = (r0 * fo[i]) / sm;
        }
#pragma unroll
        for (int i = 1; i < NQ7; ++i)
            if (fo[i] < R(0)) {
                const R a = -fo[i];
                fo[opp7(i)] = fo[opp7(i)] + a;
                fo[i] = R(0);
                added = added + R(2) * a;
            }
    } else {
        R r0 = fo[0];
#pragma unroll
        for (int i = 1; i < NQ7; ++i) r0 = r0 + fo[i];
#pragma unroll
        for (int i = 0; i < NQ7; ++i)
            if (fo[i] < R(0)) fo[i] = R(0);
        R sm = fo[0];
#pragma unroll
        for (int i = 1; i < NQ7; ++i) sm = sm + fo[i];
#pragma unroll
        for (int i = 0; i < NQ7; ++i) fo[i] = (r0 * fo[i]) / sm;
    }
    return added;
}

// For the TMA-staged D2Q7 update (as division_record for D2Q9): where
// division e goes. Its node's tile (of kTmaBoxX x 2^upd_tyl2 nodes of the
// active window, dealt round-robin over upd_ctas CTAs), that tile's index
// among the owner's tiles, and the offsets of its two pre-stream slots in the
// tile's staged box ((kTmaBoxX + 8) x (2^upd_tyl2 + 2) x 7 with the tile at
// column 4, row 1): the source (x + src7_dx(q, y & 1), y + src7_dy(q)),
// unwrapped in x (the box holds the ghost columns -1 and W), or across a wall
// the node's own population opp7(q). Returns the owner CTA.
__device__ __forceinline__ int division_record7(const SimDev &d, int e, uint32_t key, int y_r)
{
    constexpr int LX = kTmaBoxX + 8;
    const int TY = 1 << d.upd_tyl2, PL = (TY + 2) * LX;
    const int x = key_x(key), y = key_y(key), p = key_pair(key);
    const int ncx = (d.W + kTmaBoxX - 1) / kTmaBoxX;
    const int ty = (y - y_r) >> d.upd_tyl2, tx = x / kTmaBoxX;
    const uint32_t tile = (uint32_t)(ty * ncx + tx);
    const uint32_t q = __umulhi(tile, d.upd_magic);
    const int x0 = tx * kTmaBoxX, y0 = y_r + ty * TY;
    const int owner = (int)(tile - q * (uint32_t)d.upd_ctas);
    d.rec_owner[e] = owner;
    d.rec_k[e] = (int)q;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int qd = h == 0 ? Lat7::pa(p) : Lat7::pb(p);
        const int ys = y + src7_dy(qd);
        d.rec_off[2 * e + h] = (ys < y_r || ys >= d.H)
                                   ? opp7(qd) * PL + (y - y0 + 1) * LX + (x - x0 + 4)
                                   : qd * PL + (ys - y0 + 1) * LX + (x + src7_dx(qd, y & 1) - x0 + 4);
    }
    return owner;
}

// ===========================================================================
// The fused update on D2Q7 (App. A steps 1, 2, 4-7; step 3's divisions were
// added to the pre-stream slots by k_inject): as update_body, with the
// parity-dependent streaming of the triangular lattice. Blocks blk = 0 ..
// nblk - 1 (a multiple of the column tiles) of TPB threads, NR rows each.
template <typename S, int TPB, int NR>
__device__ __forceinline__ void update7_body(const SimDev &d, int blk, int nblk)
{
    using R = S;
    const uint32_t t = (uint32_t)d.sc->step;
    const int cur = (int)(t & 1u);
    const S *__restrict__ fin = (const S *)d.f[cur];
    S *__restrict__ fout = (S *)d.f[cur ^ 1];
    const int y_r = d.sc->y_r, y_copy = d.sc->y_copy, y_hi = d.sc->y_hi;
    const int W = d.W, H = d.H, Wp = d.Wp;
    const long long P = d.P;
    const int lane = threadIdx.x & 31;

    // rows the rear wall has just frozen: bring this copy up to date
    if (y_copy < y_r) {
        const long long n = (long long)(y_r - y_copy) * Wp;
        for (long long k = (long long)blk * TPB + threadIdx.x; k < n; k += (long long)nblk * TPB) {
            const long long o = (long long)y_copy * Wp + k - kXO;
#pragma unroll
            for (int i = 0; i < NQ7; ++i) fout[i * P + o] = fin[i * P + o];
        }
    }

    const R rho_c = rho_c_of<R>(d);
    const Consts<R> cf = make_consts<R>(d);
    const bool periodic = d.y_periodic != 0;
    const int ncx = (W + TPB - 1) / TPB;
    const int nrows = y_hi - y_r;
    long long mass = 0;
    int maxrow = -1;
    R clip = R(0);
    if (nrows > 0) {
        const int nty = (nrows + NR - 1) / NR;
        const int tx = blk % ncx;
        const int ty_step = nblk / ncx;
        for (int ty = blk / ncx; ty < nty; ty += ty_step) {
            const int x = tx * TPB + threadIdx.x;
            const bool colok = x < W;
            const int xm = x == 0 ? W - 1 : x - 1;
            const int xp = x >= W - 1 ? 0 : x + 1;
            R fs[NR][NQ7];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int y = y_r + ty * NR + r;
#pragma unroll
                for (int i = 0; i < NQ7; ++i) fs[r][i] = R(0);
                if (y < y_hi && colok) {
                    const bool bb_lo = !periodic && y - 1 < y_r;
                    const bool bb_hi = !periodic && y + 1 >= H;
                    const int ym = periodic ? (y == 0 ? H - 1 : y - 1) : y - 1;
                    const int yp = periodic ? (y == H - 1 ? 0 : y + 1) : y + 1;
                    const bool odd = (y & 1) != 0;
                    // the neighbours between rows: lower/upper left (x - 1 on
                    // even rows, x on odd) and right (x on even, x + 1 on odd)
                    const int xl = odd ? x : xm, xr = odd ? xp : x;
                    const S *rc = fin + (long long)y * Wp;
                    const S *rm = fin + (long long)ym * Wp;
                    const S *rp = fin + (long long)yp * Wp;
                    fs[r][0] = rc[x];
                    fs[r][1] = rc[P + xm];
                    fs[r][4] = rc[4 * P + xp];
                    if (bb_lo) { // half-way bounce-back: the node's own opposite
                        fs[r][2] = rc[5 * P + x];
                        fs[r][3] = rc[6 * P + x];
                    } else {
                        fs[r][2] = rm[2 * P + xl];
                        fs[r][3] = rm[3 * P + xr];
                    }
                    if (bb_hi) {
                        fs[r][5] = rc[2 * P + x];
                        fs[r][6] = rc[3 * P + x];
                    } else {
                        fs[r][5] = rp[5 * P + xr];
                        fs[r][6] = rp[6 * P + xl];
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int y = y_r + ty * NR + r;
                if (y >= y_hi) break; // uniform across the block
                const R *g = fs[r];
                R rho = g[0];
#pragma unroll
                for (int i = 1; i < NQ7; ++i) rho = rho + g[i];
                const bool occ = colok && rho >= rho_c;
                R fo[NQ7];
                R added = R(0);
                if (occ) {
                    R eta[NQ7];
                    if (d.noise_on) {
                        noise_eta7<R>(eta, philox4x32_10(u32x4{(uint32_t)(y * W + x), t, STREAM_NOISE, d.sim}, d.pk),
                                      cf);
                        collide7<R>(g, rho, fo, cf, eta);
                    } else {
                        collide7<R>(g, rho, fo, cf, nullptr);
                    }
                    added = fix_negative7<R>(fo, d.negfix);
                    clip += added;
                } else {
                    // rho < rho_c: reverse the directions (two-step bounce-back)
#pragma unroll
                    for (int i = 0; i < NQ7; ++i) fo[i] = g[opp7(i)];
                }
                const unsigned bits = __ballot_sync(0xffffffffu, occ);
                const int wx0 = x - lane;
                if (lane == 0 && wx0 < W) d.mask[(long long)y * d.MW + (wx0 >> 5)] = bits;
                if (colok) {
                    S *o = fout + (long long)y * Wp + x;
#pragma unroll
                    for (int i = 0; i < NQ7; ++i) o[i * P] = fo[i];
                    // the ghost copies of the edge columns
                    if (x == 0) {
#pragma unroll
                        for (int i = 0; i < NQ7; ++i) o[i * P + W] = fo[i];
                    }
                    if (x == W - 1) {
#pragma unroll
                        for (int i = 0; i < NQ7; ++i) o[i * P - W] = fo[i];
                    }
                    // the node's mass: FP64 the stored sum in index order (as
                    // the oracle); FP32 rho plus what the fix added
                    R ro;
                    if constexpr (sizeof(R) == 8) {
                        ro = fo[0];
#pragma unroll
                        for (int i = 1; i < NQ7; ++i) ro = ro + fo[i];
                    } else {
                        ro = rho + added;
                    }
                    mass += fix24<R>(ro);
                    if (ro != R(0)) maxrow = y;
                }
            }
        }
    }
    mass = warp_sum_ll(mass);
    maxrow = warp_max_i(maxrow);
    const double clipd = warp_sum_d((double)clip);
    if (lane == 0) {
        if (mass != 0) atomicAdd(&d.sc->mass_accum, (unsigned long long)mass);
        if (maxrow >= 0) atomicMax(&d.sc->maxmass_accum, maxrow);
        if (clipd != 0.0) atomicAdd(&d.sc->clip_mass, clipd);
    }
}

template <typename S, int TPB, int NR>
__global__ void __launch_bounds__(TPB) k_update7(SimDev d)
{
    update7_body<S, TPB, NR>(d, (int)blockIdx.x, (int)gridDim.x);
}

template <typename S, int TPB, int NR>
__global__ void __launch_bounds__(TPB) k_update7_batch(const SimDev *__restrict__ ds, const int4 *__restrict__ bm)
{
    const int4 a = bm[blockIdx.x];
    if (a.x < 0) return; // an unused entry
    update7_body<S, TPB, NR>(ds[a.x], a.y, a.z);
}

} // namespace lbm
