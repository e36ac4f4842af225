// Kernels of the growing-tissue LBM hot path, templated on the population
// storage type R (float: fast path; double: debug path, compiled without FMA
// contraction so that it rounds exactly like the FP64 CPU oracle).
//
// One time step (App. A of Killeen et al., arXiv 2303.02210) is two launches:
//   k_update  the fused pass over the active window: pull streaming with
//             half-way bounce-back walls, moments (Eq. 1), friction u*, f^SS
//             (Eq. 3), BGK relaxation or reversal below rho_c (Eq. 2 and the
//             two-step bounce-back of Sec. II), Philox noise (Eq. 4), the
//             negative-population fix (App. A step 7), the store, the occupancy
//             bitmask (one warp ballot per 32 nodes) and the exact fixed-point
//             mass / top-mass-row reductions (k_update_tma, lbm_update_tma.cuh,
//             is the TMA-staged FP32 form);
//   k_plan    (lbm_plan.cuh) the observables of the new state and the
//             proliferation of the next step: front heights, Eq. 6, the rear
//             wall, n_s, candidate draws, acceptance, selection and merge,
//             injection (or records for k_update_tma).
#pragma once

#include "lbm_common.cuh"

namespace lbm {

template <typename R>
__device__ __forceinline__ long long fix24(R r);
// FP32: v = r * 2^24 is exact, and v >= 0 (populations are non-negative).
// Below 2^23 the add of 2^23 rounds v to the nearest integer (ties to even)
// in the mantissa; from 2^23 on v is already an integer and its bits give it
// directly. No conversion instruction (those run on a slow pipe).
template <>
__device__ __forceinline__ long long fix24<float>(float r)
{
    const float v = r * 16777216.0f;
    const long long lo = (long long)(__float_as_uint(v + 8388608.0f) - 0x4B000000u);
    const uint32_t b = __float_as_uint(v);
    const long long hi = (long long)((unsigned long long)((b & 0x7FFFFFu) | 0x800000u) << ((b >> 23) - 150u));
    return v < 8388608.0f ? lo : hi; // v < 2^63 always (rho < 2^39)
}
template <>
__device__ __forceinline__ long long fix24<double>(double r) { return __double2ll_rn(r * 16777216.0); }

// Occupancy threshold in the storage type (the FP32 copy is rounded on the host).
template <typename R>
__device__ __forceinline__ R rho_c_of(const SimDev &d)
{
    if constexpr (sizeof(R) == 8)
        return d.rho_c;
    else
        return d.f_rho_c;
}

// ===========================================================================
// Population storage. FP32 and FP64 hold f_i as it is and compute in the
// same type. The 16-bit forms (FP16, BF16) hold the deviation f_i - c_i from
// the rest state of density rho_init, c_i = w_i rho_init rounded to the
// 16-bit type, and compute in FP32: decode is float(s) + c_i, encode rounds
// f_i - c_i to nearest. Because c_i is itself a 16-bit value, f_i = 0 (the
// void) and f_i = c_i are both stored exactly, and rounding is monotone, so
// a non-negative f_i never decodes below zero. c_i depends only on the
// weight class of i, which i and opp(i) share, so a bounce-back load may
// decode with the class of the plane it reads.
__host__ __device__ constexpr int wclass(int q) { return q == 0 ? 0 : (q < 5 ? 1 : 2); }

template <typename S>
struct Pop {
    using R = S; // arithmetic type
    static constexpr bool kShifted = false;
    __device__ explicit Pop(const SimDev &) {}
    __device__ explicit Pop(const float *) {} // (from the three shifts)
    __device__ R ld(S v, int) const { return v; }
    __device__ S st(R v, int) const { return v; }
};

template <typename S, typename Cvt>
struct PopShifted {
    using R = float;
    static constexpr bool kShifted = true;
    float c0, c1, c2;
    __device__ explicit PopShifted(const SimDev &d) : c0(d.pop_shift[0]), c1(d.pop_shift[1]), c2(d.pop_shift[2]) {}
    __device__ explicit PopShifted(const float *sh) : c0(sh[0]), c1(sh[1]), c2(sh[2]) {}
    __device__ float shift(int q) const
    {
        const int k = wclass(q);
        return k == 0 ? c0 : (k == 1 ? c1 : c2);
    }
    __device__ float ld(S v, int q) const { return Cvt::add(v, shift(q)); }
    __device__ S st(float v, int q) const { return Cvt::from_f(v - shift(q)); }
};
// add(v, s) = to_f(v) + s. BF16: one mixed-precision add (sm_100 and later;
// the 16-bit operand is widened exactly and the sum rounded once to nearest
// in FP32, the same value as the conversion followed by an FP32 add), which
// measured 0.7% faster per update than the conversion and add at 8192 x 2048;
// FP16 keeps the conversion and add (the mixed add measured 2.4% slower).
struct CvtHalf {
    static __device__ float to_f(__half v) { return __half2float(v); }
    static __device__ __half from_f(float v) { return __float2half_rn(v); }
    static __device__ float add(__half v, float s) { return __half2float(v) + s; }
};
struct CvtBf16 {
    static __device__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __nv_bfloat16 from_f(float v) { return __float2bfloat16_rn(v); }
    static __device__ float add(__nv_bfloat16 v, float s)
    {
        float r;
        asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(r) : "h"(__bfloat16_as_ushort(v)), "f"(s));
        return r;
    }
};
template <>
struct Pop<__half> : PopShifted<__half, CvtHalf> {
    __device__ explicit Pop(const SimDev &d) : PopShifted<__half, CvtHalf>(d) {}
    __device__ explicit Pop(const float *sh) : PopShifted<__half, CvtHalf>(sh) {}
};
template <>
struct Pop<__nv_bfloat16> : PopShifted<__nv_bfloat16, CvtBf16> {
    __device__ explicit Pop(const SimDev &d) : PopShifted<__nv_bfloat16, CvtBf16>(d) {}
    __device__ explicit Pop(const float *sh) : PopShifted<__nv_bfloat16, CvtBf16>(sh) {}
};
template <typename S>
using arith_t = typename Pop<S>::R;

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_max_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_min_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Index of the pre-stream slot that streams into direction d of node (x, y):
// the neighbour (x - ex_d, y - ey_d), or, across a wall, the node's own
// opposite population (half-way bounce-back).
__device__ __forceinline__ long long pull_slot(const SimDev &d, int y_r, int x, int y, int q)
{
    int ys = y - ey(q);
    if (d.y_periodic) {
        ys = ys < 0 ? ys + d.H : (ys >= d.H ? ys - d.H : ys);
    } else if (ys < y_r || ys >= d.H) {
        return (long long)opp(q) * d.P + (long long)y * d.Wp + x;
    }
    int xs = x - ex(q);
    xs = xs < 0 ? xs + d.W : (xs >= d.W ? xs - d.W : xs);
    return (long long)q * d.P + (long long)ys * d.Wp + xs;
}

// ---------------------------------------------------------------------------
// What the planner needs to know about a lattice: its directions, the
// pre-stream slot of a direction, and the opposite pairs a division loads.
// Lat9: D2Q9. Lat7: the triangular D2Q7 (Sec. II) with rows of nodes along
// x, odd rows shifted by half a spacing: 1:(1,0) 2:(1/2,s) 3:(-1/2,s)
// 4:(-1,0) 5:(-1/2,-s) 6:(1/2,-s), s = sqrt(3)/2; opp(q) = q + 3 (mod 6);
// the neighbour of (x, y) along 2 is (x + (y & 1), y + 1).
struct Lat9 {
    static constexpr int Q = 9;
    __device__ static long long slot(const SimDev &d, int y_r, int x, int y, int q)
    {
        return pull_slot(d, y_r, x, y, q);
    }
    __device__ static int pair_of(uint32_t r) { return (int)(r >> 30); }
    __device__ static int pa(int p) { return pair_a(p); }
    __device__ static int pb(int p) { return pair_b(p); }
};

__host__ __device__ constexpr int opp7(int q) { return q == 0 ? 0 : (q <= 3 ? q + 3 : q - 3); }
// source of direction q at (x, y) before any wrap or wall: x offset by row
// parity for the directions between rows
__host__ __device__ constexpr int src7_dx(int q, int par)
{
    return q == 1 ? -1 : (q == 4 ? 1 : (q == 2 || q == 6 ? par - 1 : (q == 3 || q == 5 ? par : 0)));
}
__host__ __device__ constexpr int src7_dy(int q) { return q == 2 || q == 3 ? -1 : (q == 5 || q == 6 ? 1 : 0); }

struct Lat7 {
    static constexpr int Q = 7;
    __device__ static long long slot(const SimDev &d, int y_r, int x, int y, int q)
    {
        int ys = y + src7_dy(q);
        if (d.y_periodic) {
            ys = ys < 0 ? ys + d.H : (ys >= d.H ? ys - d.H : ys);
        } else if (ys < y_r || ys >= d.H) {
            return (long long)opp7(q) * d.P + (long long)y * d.Wp + x;
        }
        int xs = x + src7_dx(q, y & 1);
        xs = xs < 0 ? xs + d.W : (xs >= d.W ? xs - d.W : xs);
        return (long long)q * d.P + (long long)ys * d.Wp + xs;
    }
    // a pair uniform over the three
    __device__ static int pair_of(uint32_t r) { return (int)(((unsigned long long)r * 3ull) >> 32); }
    __device__ static int pa(int p) { return p + 1; }
    __device__ static int pb(int p) { return p + 4; }
};

// ===========================================================================
// Initial state (App. A, first paragraph): rho = rho_init (optionally
// jittered by U[1 - j, 1 + j]) below the front, zero above, u = 0,
// f_i = f^SS_i(rho, 0) = w_i rho. Written into both population copies.
template <typename S>
__global__ void k_fill(SimDev d)
{
    using R = arith_t<S>;
    const Pop<S> pc(d);
    S *f0 = (S *)d.f[0];
    S *f1 = (S *)d.f[1];
    if (blockIdx.x == 0 && threadIdx.x == 0) { // scalar block (zeroed before this launch)
        d.sc->maxmass_accum = -1;
        d.sc->low_acc = 0x7fffffff;
    }
    // every stored element of a row: x = -kXO .. Wp - kXO - 1; the ghost
    // columns x = -1 and x = W take the values of x = W - 1 and x = 0
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
        for (int i = 0; i < NQ; ++i) {
            const S v = pc.st((R)(wq<double>(i) * rho), i);
            f0[i * d.P + o] = v;
            f1[i * d.P + o] = v;
        }
    }
}

// Ghost columns x = -1 and x = W of every row of both copies from columns
// W - 1 and 0 (after the caller has written the populations).
template <typename S>
__global__ void k_ghosts(SimDev d)
{
    const long long total = 2LL * NQ * d.H;
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

// Occupancy mask, exact mass and highest mass row of rows [y_r, H) of copy
// `cur` (initial state, or populations set by the caller).
template <typename S>
__global__ void k_scan(SimDev d, int cur)
{
    using R = arith_t<S>;
    const Pop<S> pc(d);
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
            rho = pc.ld(f[n], 0);
            any = rho != R(0);
#pragma unroll
            for (int i = 1; i < NQ; ++i) {
                const R v = pc.ld(f[i * d.P + n], i);
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

// ===========================================================================
// Per-node collision pieces of the update kernel.
//
// FP64 (debug path): every formula in the order of the CPU oracle, so the
// results agree bit for bit. FP32 (fast path): the same quantities, regrouped
// (algebraically identical in exact arithmetic) for fewer instructions:
//  * u* = (1 - mu) j / rho with one reciprocal;
//  * Eq. 3 by opposite pairs: with p = 1 - 3/2 u*.u* + 9/2 (e.u*)^2, the
//    factor is p + 3 e.u* for e and p - 3 e.u* for -e;
//  * f_0 = rho - sum_{i>0} f_i, i.e. the BGK step's exact mass conservation
//    (sum_i w_i (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u) = 1), which keeps the
//    rounding of the float weights from drifting the total mass;
//  * the noise uniforms built from mantissa bits (no integer conversions).
template <typename R>
struct Consts {
    R omega, cmu, om1, ow0, ow1, ow5, two_sigma;
};

template <typename R>
__device__ __forceinline__ Consts<R> make_consts(const SimDev &d)
{
    Consts<R> c;
    if constexpr (sizeof(R) == 8) {
        c.omega = d.omega;
        c.cmu = d.cmu;
        c.om1 = 1.0 - d.omega;
        c.ow0 = d.omega * (4.0 / 9.0);
        c.ow1 = d.omega * (1.0 / 9.0);
        c.ow5 = d.omega * (1.0 / 36.0);
        c.two_sigma = 2.0 * d.sigma;
    } else {
        c.omega = d.f_omega;
        c.cmu = d.f_cmu;
        c.om1 = d.f_om1;
        c.ow0 = d.f_ow0;
        c.ow1 = d.f_ow1;
        c.ow5 = d.f_ow5;
        c.two_sigma = d.f_two_sigma;
    }
    return c;
}

template <typename R>
__device__ __forceinline__ void collide(const R *g, R rho, R *fo, const Consts<R> &c, const R *eta)
{
    const R jx = ((((g[1] - g[3]) + g[5]) - g[6]) - g[7]) + g[8];
    const R jy = ((((g[2] - g[4]) + g[5]) + g[6]) - g[7]) - g[8];
    if constexpr (sizeof(R) == 8) {
        const R ux = jx / rho, uy = jy / rho;
        const R usx = c.cmu * ux, usy = c.cmu * uy; // u* = (1 - mu) u
        const R uu = usx * usx + usy * usy;
        const R eu[NQ] = {R(0), usx, usy, -usx, -usy, usx + usy, -usx + usy, -usx - usy, usx - usy};
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            R t1 = R(1) + R(3) * eu[i];
            t1 = t1 + R(4.5) * (eu[i] * eu[i]);
            t1 = t1 - R(1.5) * uu;
            const R fss = (wq<R>(i) * rho) * t1;    // Eq. 3, D2Q9
            fo[i] = g[i] - c.omega * (g[i] - fss); // Eq. 2
        }
        if (eta) {
#pragma unroll
            for (int i = 0; i < NQ; ++i) fo[i] = fo[i] + eta[i]; // Eq. 4
        }
    } else {
        float rr;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rr) : "f"(rho));
        const float k = c.cmu * rr;
        const float usx = jx * k, usy = jy * k;
        const float A = fmaf(-1.5f, fmaf(usx, usx, usy * usy), 1.0f);
        const float r1 = c.ow1 * rho, r5 = c.ow5 * rho;
        // every multiply-add is an explicit fmaf, so the rounding does not
        // depend on the compiler's contraction choices; the noise rides in
        // the innermost one
        float e, p;
        e = usx;
        p = fmaf(4.5f * e, e, A);
        fo[1] = fmaf(c.om1, g[1], fmaf(r1, fmaf(3.0f, e, p), eta[1]));
        fo[3] = fmaf(c.om1, g[3], fmaf(r1, fmaf(-3.0f, e, p), eta[3]));
        e = usy;
        p = fmaf(4.5f * e, e, A);
        fo[2] = fmaf(c.om1, g[2], fmaf(r1, fmaf(3.0f, e, p), eta[2]));
        fo[4] = fmaf(c.om1, g[4], fmaf(r1, fmaf(-3.0f, e, p), eta[4]));
        e = usx + usy;
        p = fmaf(4.5f * e, e, A);
        fo[5] = fmaf(c.om1, g[5], fmaf(r5, fmaf(3.0f, e, p), eta[5]));
        fo[7] = fmaf(c.om1, g[7], fmaf(r5, fmaf(-3.0f, e, p), eta[7]));
        e = usy - usx;
        p = fmaf(4.5f * e, e, A);
        fo[6] = fmaf(c.om1, g[6], fmaf(r5, fmaf(3.0f, e, p), eta[6]));
        fo[8] = fmaf(c.om1, g[8], fmaf(r5, fmaf(-3.0f, e, p), eta[8]));
        // f_0 = rho - sum_{i>0} f_i: BGK (Eq. 2) and the noise (Eq. 4) both
        // conserve the node's mass exactly, so this is f_0 in exact
        // arithmetic, and it keeps the rounding of the float weights and of
        // 1/9 from drifting the total mass
        fo[0] = rho - ((((fo[1] + fo[2]) + (fo[3] + fo[4])) + ((fo[5] + fo[6]) + (fo[7] + fo[8]))));
    }
}

// The nine 14-bit fields of a Philox block read as one 128-bit integer
// w.x + 2^32 w.y + 2^64 w.z + 2^96 w.w: field i is bits 14 i .. 14 i + 13.
__device__ __forceinline__ void noise_fields(const u32x4 &w, uint32_t m[NQ])
{
    m[0] = w.x;
    m[1] = w.x >> 14;
    m[2] = __funnelshift_r(w.x, w.y, 28);
    m[3] = w.y >> 10;
    m[4] = __funnelshift_r(w.y, w.z, 24);
    m[5] = w.z >> 6;
    m[6] = __funnelshift_r(w.z, w.w, 20);
    m[7] = w.w >> 2;
    m[8] = w.w >> 16;
#pragma unroll
    for (int i = 0; i < NQ; ++i) m[i] &= 0x3FFFu;
}

// Eq. 4: eta_i = 2 sigma (u_i - mean u), u_i = (m_i + 1/2) 2^-14 with m_i the
// 14-bit fields of the node's Philox block (n, t, 16, sim), given as `w`.
template <typename R>
__device__ __forceinline__ void noise_eta_words(R *eta, const u32x4 &w, const Consts<R> &c)
{
    uint32_t m[NQ];
    noise_fields(w, m);
    if constexpr (sizeof(R) == 8) {
        double u[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) u[i] = ((double)m[i] + 0.5) * 6.103515625e-05;
        double S = u[0];
#pragma unroll
        for (int i = 1; i < NQ; ++i) S = S + u[i];
        const double ubar = S / 9.0;
#pragma unroll
        for (int i = 0; i < NQ; ++i) eta[i] = c.two_sigma * (u[i] - ubar);
    } else {
        // 1 + m 2^-14 exactly; the constant offset cancels in u_i - mean u
        float v[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) v[i] = __uint_as_float(0x3F800000u | (m[i] << 9));
        const float S = (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) + v[8];
        const float nb = -c.two_sigma * (S * (1.0f / 9.0f));
        eta[0] = 0.0f; // f_0 follows from mass conservation
#pragma unroll
        for (int i = 1; i < NQ; ++i) eta[i] = fmaf(c.two_sigma, v[i], nb);
    }
}

// The noise block of node n at step t.
__device__ __forceinline__ u32x4 noise_block(uint32_t n, uint32_t t, const SimDev &d)
{
    return philox4x32_10(u32x4{n, t, STREAM_NOISE, d.sim}, d.pk);
}

template <typename R>
__device__ __forceinline__ void noise_eta(R *eta, uint32_t n, uint32_t t, const SimDev &d, const Consts<R> &c)
{
    noise_eta_words<R>(eta, noise_block(n, t, d), c);
}

template <typename R>
__device__ __forceinline__ R fix_negative(R *fo, int mode);

// One occupied node: Eq. 3 / Eq. 2 relaxation with (NOISE) the Eq. 4 noise,
// before the negative-population fix.
template <typename R, bool NOISE>
__device__ __forceinline__ void relax_core(const R *g, R rho, R *fo, uint32_t n, uint32_t t, const SimDev &d,
                                           const Consts<R> &c)
{
    R eta[NQ];
    if constexpr (NOISE) {
        noise_eta<R>(eta, n, t, d, c);
    } else {
#pragma unroll
        for (int i = 0; i < NQ; ++i) eta[i] = R(0);
    }
    if constexpr (sizeof(R) == 8)
        collide<R>(g, rho, fo, c, NOISE ? eta : nullptr);
    else
        collide<R>(g, rho, fo, c, eta);
}

// relax_core with the node's noise block already drawn (`w`, unused without noise).
template <typename R, bool NOISE>
__device__ __forceinline__ void relax_words(const R *g, R rho, R *fo, const u32x4 &w, const Consts<R> &c)
{
    R eta[NQ];
    if constexpr (NOISE) {
        noise_eta_words<R>(eta, w, c);
    } else {
#pragma unroll
        for (int i = 0; i < NQ; ++i) eta[i] = R(0);
    }
    if constexpr (sizeof(R) == 8)
        collide<R>(g, rho, fo, c, NOISE ? eta : nullptr);
    else
        collide<R>(g, rho, fo, c, eta);
}

// relax_core followed by the negative-population fix. Returns the mass the
// fix added.
template <typename R>
__device__ __forceinline__ R relax_node(const R *g, R rho, R *fo, uint32_t n, uint32_t t, const SimDev &d,
                                        const Consts<R> &c)
{
    if (d.noise_on)
        relax_core<R, true>(g, rho, fo, n, t, d, c);
    else
        relax_core<R, false>(g, rho, fo, n, t, d, c);
    return fix_negative<R>(fo, d.negfix);
}

// Mass of the stored populations of a node. FP64 (as the oracle): their sum
// in index order. FP32: the node's density before the update plus what the
// negative-population fix added, which is that sum in exact arithmetic (the
// update and the reversal conserve mass).
template <typename R>
__device__ __forceinline__ R node_mass(const R *fo, R rho, R added)
{
    if constexpr (sizeof(R) == 8) {
        R r = fo[0];
#pragma unroll
        for (int i = 1; i < NQ; ++i) r = r + fo[i];
        return r;
    } else {
        return rho + added;
    }
}

// App. A step 7: negative-population correction. Returns the mass it adds.
template <typename R>
__device__ __forceinline__ R fix_negative(R *fo, int mode)
{
    R added = R(0);
    if constexpr (sizeof(R) == 4) {
        const float mn = fminf(fminf(fminf(fo[0], fo[1]), fminf(fo[2], fo[3])),
                               fminf(fminf(fo[4], fo[5]), fminf(fminf(fo[6], fo[7]), fo[8])));
        if (mn >= 0.0f) return added; // the common case
    }
    if (mode == 0) {
        if (fo[0] < R(0)) {
            R r0 = fo[0];
#pragma unroll
            for (int i = 1; i < NQ; ++i) r0 = r0 + fo[i];
            fo[0] = R(0);
            R sm = fo[0];
#pragma unroll
            for (int i = 1; i < NQ; ++i) sm = sm + fo[i];
#pragma unroll
            for (int i = 0; i < NQ; ++i) fo[i] = (r0 * fo[i]) / sm;
        }
#pragma unroll
        for (int i = 1; i < NQ; ++i) {
            if (fo[i] < R(0)) {
                const R a = -fo[i];
                fo[opp(i)] = fo[opp(i)] + a;
                fo[i] = R(0);
                added += a + a;
            }
        }
    } else {
        bool neg = false;
#pragma unroll
        for (int i = 0; i < NQ; ++i) neg |= fo[i] < R(0);
        if (neg) {
            R r0 = fo[0];
#pragma unroll
            for (int i = 1; i < NQ; ++i) r0 = r0 + fo[i];
#pragma unroll
            for (int i = 0; i < NQ; ++i) fo[i] = fo[i] < R(0) ? R(0) : fo[i];
            R sm = fo[0];
#pragma unroll
            for (int i = 1; i < NQ; ++i) sm = sm + fo[i];
#pragma unroll
            for (int i = 0; i < NQ; ++i) fo[i] = (r0 * fo[i]) / sm;
        }
    }
    return added;
}

// ===========================================================================
// Fused update of the active window (App. A steps 1, 2, 4-7; the injection of
// step 3 was already added to the pre-stream slots by k_inject), run by blocks
// blk = 0 .. nblk - 1 of TPB threads.
template <typename S, int TPB, int NR>
__device__ __forceinline__ void update_body(const SimDev &d, int blk, int nblk)
{
    using R = arith_t<S>;
    const Pop<S> pc(d);
    // the step is read from the device (so a captured step replays as is):
    // step t reads copy t & 1
    const uint32_t t = (uint32_t)d.sc->step;
    const int cur = (int)(t & 1u);
    const S *__restrict__ fin = (const S *)d.f[cur];
    S *__restrict__ fout = (S *)d.f[cur ^ 1];
    const int y_r = d.sc->y_r, y_copy = d.sc->y_copy, y_hi = d.sc->y_hi;
    const int W = d.W, H = d.H, Wp = d.Wp;
    const long long P = d.P;
    const int lane = threadIdx.x & 31;

    // Rows the rear wall has just frozen: bring this copy up to date.
    if (y_copy < y_r) {
        const long long n = (long long)(y_r - y_copy) * Wp;
        for (long long k = (long long)blk * TPB + threadIdx.x; k < n; k += (long long)nblk * TPB) {
            const long long o = (long long)y_copy * Wp + k - kXO; // whole stored rows, ghosts included
#pragma unroll
            for (int i = 0; i < NQ; ++i) fout[i * P + o] = fin[i * P + o];
        }
    }

    const R rho_c = rho_c_of<R>(d);
    const Consts<R> cf = make_consts<R>(d);
    const bool periodic = d.y_periodic != 0;
    const int ncx = (W + TPB - 1) / TPB;
    const int nrows = y_hi - y_r;
    long long mass = 0;
    int maxrow = -1;
    R clip = R(0); // mass added by the negative-population fix, this thread
    if (nrows > 0) {
        // the grid is a multiple of the column-tile count: each block keeps
        // one column tile and strides over the rows
        const int nty = (nrows + NR - 1) / NR;
        const int tx = blk % ncx;
        const int ty_step = nblk / ncx;
        for (int ty = blk / ncx; ty < nty; ty += ty_step) {
            const int x = tx * TPB + threadIdx.x;
            const bool colok = x < W;
            const int xm = x == 0 ? W - 1 : x - 1;
            const int xp = x >= W - 1 ? 0 : x + 1;
            R fs[NR][NQ];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int y = y_r + ty * NR + r;
#pragma unroll
                for (int i = 0; i < NQ; ++i) fs[r][i] = R(0);
                if (y < y_hi && colok) {
                    const bool bb_lo = !periodic && y - 1 < y_r;
                    const bool bb_hi = !periodic && y + 1 >= H;
                    const int ym = periodic ? (y == 0 ? H - 1 : y - 1) : y - 1;
                    const int yp = periodic ? (y == H - 1 ? 0 : y + 1) : y + 1;
                    const S *rc = fin + (long long)y * Wp;
                    const S *rm = fin + (long long)ym * Wp;
                    const S *rp = fin + (long long)yp * Wp;
                    // (a bounce-back load decodes with the class of the plane
                    // it reads, which is the class of the one it fills)
                    fs[r][0] = pc.ld(rc[x], 0);
                    fs[r][1] = pc.ld(rc[P + xm], 1);
                    fs[r][3] = pc.ld(rc[3 * P + xp], 3);
                    if (bb_lo) {
                        fs[r][2] = pc.ld(rc[4 * P + x], 4);
                        fs[r][5] = pc.ld(rc[7 * P + x], 7);
                        fs[r][6] = pc.ld(rc[8 * P + x], 8);
                    } else {
                        fs[r][2] = pc.ld(rm[2 * P + x], 2);
                        fs[r][5] = pc.ld(rm[5 * P + xm], 5);
                        fs[r][6] = pc.ld(rm[6 * P + xp], 6);
                    }
                    if (bb_hi) {
                        fs[r][4] = pc.ld(rc[2 * P + x], 2);
                        fs[r][7] = pc.ld(rc[5 * P + x], 5);
                        fs[r][8] = pc.ld(rc[6 * P + x], 6);
                    } else {
                        fs[r][4] = pc.ld(rp[4 * P + x], 4);
                        fs[r][7] = pc.ld(rp[7 * P + xp], 7);
                        fs[r][8] = pc.ld(rp[8 * P + xm], 8);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int y = y_r + ty * NR + r;
                if (y >= y_hi) break; // uniform across the block
                const R *g = fs[r];
                // Eq. 1 on f*: density in index order
                R rho = g[0];
#pragma unroll
                for (int i = 1; i < NQ; ++i) rho = rho + g[i];
                const bool occ = colok && rho >= rho_c;
                R fo[NQ];
                R added = R(0);
                if (occ) {
                    added = relax_node<R>(g, rho, fo, (uint32_t)(y * W + x), t, d, cf);
                    clip += added;
                } else {
                    // rho < rho_c: reverse the directions (two-step bounce-back)
#pragma unroll
                    for (int i = 0; i < NQ; ++i) fo[i] = g[opp(i)];
                }
                const unsigned bits = __ballot_sync(0xffffffffu, occ);
                const int wx0 = x - lane;
                if (lane == 0 && wx0 < W) d.mask[(long long)y * d.MW + (wx0 >> 5)] = bits;
                if (colok) {
                    S *o = fout + (long long)y * Wp + x;
                    R ro;
                    if constexpr (Pop<S>::kShifted) {
                        // the node's mass is that of what is stored: the
                        // decoded 16-bit values, summed in index order
                        ro = R(0);
#pragma unroll
                        for (int i = 0; i < NQ; ++i) {
                            const S v = pc.st(fo[i], i);
                            o[i * P] = v;
                            ro = i == 0 ? pc.ld(v, 0) : ro + pc.ld(v, i);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < NQ; ++i) o[i * P] = fo[i];
                        ro = node_mass<R>(fo, rho, added);
                    }
                    // the ghost copies of the edge columns (stored x = W and
                    // x = -1), which the TMA-staged update reads: a lattice
                    // may be stepped by either kernel
                    if (x == 0) {
#pragma unroll
                        for (int i = 0; i < NQ; ++i) o[i * P + W] = pc.st(fo[i], i);
                    }
                    if (x == W - 1) {
#pragma unroll
                        for (int i = 0; i < NQ; ++i) o[i * P - W] = pc.st(fo[i], i);
                    }
                    // populations are non-negative after every step, so the
                    // node holds mass iff their sum is non-zero
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

// The update of one simulation: the grid is a multiple of its column tiles.
template <typename S, int TPB, int NR>
__global__ void __launch_bounds__(TPB) k_update(SimDev d)
{
    update_body<S, TPB, NR>(d, (int)blockIdx.x, (int)gridDim.x);
}

// The updates of a batch of simulations in one launch: block b works for
// simulation bm[b].x as its block bm[b].y of bm[b].z, a multiple of that
// simulation's column tiles (a table rebuilt when the members change;
// bm[b].x < 0: an unused entry, nothing to do).
template <typename S, int TPB, int NR>
__global__ void __launch_bounds__(TPB) k_update_batch(const SimDev *__restrict__ ds, const int4 *__restrict__ bm)
{
    const int4 a = bm[blockIdx.x];
    if (a.x < 0) return;
    update_body<S, TPB, NR>(ds[a.x], a.y, a.z);
}

// ===========================================================================
// Proliferation helpers (App. A step 3; Sec. II and Eq. 5), used by the fused
// planner: counter-based candidate draws (Philox (k, t, 1, sim)), the
// streamed density rho* gathered from the nine pre-stream slots, the
// open-addressing table that merges repeated (node, pair) draws, and the
// per-division records of the TMA-staged update.

template <typename S, typename LT = Lat9>
__device__ __forceinline__ arith_t<S> rho_star(const SimDev &d, const S *f, int y_r, int x, int y)
{
    using R = arith_t<S>;
    const Pop<S> pc(d);
    long long o[LT::Q];
#pragma unroll
    for (int q = 0; q < LT::Q; ++q) o[q] = LT::slot(d, y_r, x, y, q);
    R v[LT::Q];
#pragma unroll
    for (int q = 0; q < LT::Q; ++q) v[q] = pc.ld(f[o[q]], q);
    R r = v[0];
#pragma unroll
    for (int q = 1; q < LT::Q; ++q) r = r + v[q];
    return r;
}

struct Candidate {
    int x, y, pair;
    uint32_t u; // acceptance uniform word (density-dependent growth)
};

template <typename LT = Lat9>
__device__ __forceinline__ Candidate draw_candidate(const SimDev &d, long long k, uint32_t t, int ylo,
                                                    unsigned long long nwin)
{
    const u32x4 r = philox4x32_10(u32x4{(uint32_t)k, t, STREAM_PROLIF, d.sim}, d.pk);
    // node = ylo W + floor(r.x nwin / 2^32); nwin <= W H < 2^30, so the offset
    // in the window splits into row and column in 32-bit arithmetic
    const uint32_t idx = (uint32_t)(((unsigned long long)r.x * nwin) >> 32);
    Candidate c;
    c.y = ylo + (int)(idx / (uint32_t)d.W);
    c.x = (int)(idx % (uint32_t)d.W);
    c.pair = LT::pair_of(r.y);
    c.u = r.z;
    return c;
}

constexpr uint32_t EMPTY_KEY = 0xFFFFFFFFu;
constexpr unsigned long long EMPTY_ENTRY = ~0ull; // key EMPTY_KEY: never a real key

struct EventTable {
    unsigned long long *e; // (key << 32) | draw rank of the key's first draw
    unsigned mask;         // slots - 1
};

// Draw rank `rank` of `key`: returns the slot if the key is new (its entry
// then holds the key and this rank), else -1; *first is the rank of the
// key's first draw. One compare-and-swap either way.
__device__ __forceinline__ int table_insert(const EventTable &tb, uint32_t key, int rank, int *first)
{
    const unsigned long long mine = ((unsigned long long)key << 32) | (uint32_t)rank;
    unsigned slot = (unsigned)(((unsigned long long)key * 0x9E3779B97F4A7C15ull) >> 32) & tb.mask;
    for (unsigned probe = 0; probe <= tb.mask; ++probe) {
        const unsigned long long old = atomicCAS(&tb.e[slot], EMPTY_ENTRY, mine);
        if (old == EMPTY_ENTRY) {
            *first = rank;
            return (int)slot;
        }
        if ((uint32_t)(old >> 32) == key) {
            *first = (int)(uint32_t)old;
            return -1;
        }
        slot = (slot + 1u) & tb.mask;
    }
    *first = -1; // full (never: the table has at least 2 n_s,max slots)
    return -1;
}

// For the TMA-staged update: where division e goes. Its node's tile (of
// kTmaBoxX x 2^upd_tyl2 nodes of the active window; tiles are dealt
// round-robin over upd_ctas CTAs), that tile's index among the owner's tiles,
// and the offsets of the two pre-stream slots in the tile's staged box
// ((kTmaBoxX + 8) x (2^upd_tyl2 + 2) x 9 with the tile at column 4, row 1):
// the source (x - ex_q, y - ey_q) unwrapped in x (the box holds the ghost
// columns -1 and W), or across a wall the node's own population opp(q).
// Returns the owner CTA.
template <typename R>
__device__ __forceinline__ int division_record(const SimDev &d, int e, uint32_t key, int y_r)
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
        const int qd = h == 0 ? pair_a(p) : pair_b(p);
        const int ys = y - ey(qd);
        d.rec_off[2 * e + h] = (ys < y_r || ys >= d.H) ? opp(qd) * PL + (y - y0 + 1) * LX + (x - x0 + 4)
                                                       : qd * PL + (ys - y0 + 1) * LX + (x - ex(qd) - x0 + 4);
    }
    return owner;
}

// rho and u of copy `cur` into device arrays of W*H doubles (Eq. 1).
template <typename S>
__global__ void k_fields(SimDev d, int cur, double *rho, double *ux, double *uy)
{
    const Pop<S> pc(d);
    const S *f = (const S *)d.f[cur];
    const long long total = (long long)d.W * d.H;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / d.W), x = (int)(k % d.W);
        const long long o = (long long)y * d.Wp + x;
        double g[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) g[i] = (double)pc.ld(f[i * d.P + o], i);
        double r = g[0];
#pragma unroll
        for (int i = 1; i < NQ; ++i) r = r + g[i];
        const double jx = ((((g[1] - g[3]) + g[5]) - g[6]) - g[7]) + g[8];
        const double jy = ((((g[2] - g[4]) + g[5]) + g[6]) - g[7]) - g[8];
        rho[k] = r;
        ux[k] = r != 0.0 ? jx / r : 0.0;
        uy[k] = r != 0.0 ? jy / r : 0.0;
    }
}

} // namespace lbm
