// Two adjacent nodes at once: the FP32 collision, Eq. 4 noise and density sum
// of lbm_kernels.cuh written on float2 pairs (component .x the first node,
// .y the second) with Blackwell's packed FP32 instructions (add, sub, mul, fma
// on f32x2: one instruction for both nodes).
//
// Every function performs, per component, exactly the IEEE operations of its
// scalar counterpart (collide<float>, noise_eta_words<float>, the density
// sum in index order), in the same order and with the same rounding
// (round-to-nearest, no flush to zero), so a kernel built on these computes
// the same bits as one built on the scalar code.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pr, pa, pb;\n\t"
        "mov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// Eq. 1 density of the pulled populations, summed in index order.
__device__ __forceinline__ float2 rho_pair(const float2 g[NQ])
{
    float2 r = g[0];
#pragma unroll
    for (int i = 1; i < NQ; ++i) r = add2(r, g[i]);
    return r;
}

// noise_eta_words<float> for two nodes (their Philox blocks wa, wb).
__device__ __forceinline__ void noise_eta_pair(float2 eta[NQ], const u32x4 &wa, const u32x4 &wb,
                                               const Consts<float> &c)
{
    uint32_t ma[NQ], mb[NQ];
    noise_fields(wa, ma);
    noise_fields(wb, mb);
    float2 v[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i)
        v[i] = make_float2(__uint_as_float(0x3F800000u | (ma[i] << 9)), __uint_as_float(0x3F800000u | (mb[i] << 9)));
    const float2 S = add2(add2(add2(add2(v[0], v[1]), add2(v[2], v[3])), add2(add2(v[4], v[5]), add2(v[6], v[7]))),
                          v[8]);
    const float2 nb = mul2(f2(-c.two_sigma), mul2(S, f2(1.0f / 9.0f)));
    eta[0] = f2(0.0f);
#pragma unroll
    for (int i = 1; i < NQ; ++i) eta[i] = fma2(f2(c.two_sigma), v[i], nb);
}

// collide<float> for two nodes: u* = (1 - mu) j / rho with one reciprocal,
// Eq. 3 by opposite pairs, Eq. 2 relaxation with the noise in the innermost
// multiply-add, f_0 from the node's exact mass conservation.
__device__ __forceinline__ void collide_pair(const float2 g[NQ], float2 rho, float2 fo[NQ], const Consts<float> &c,
                                             const float2 eta[NQ])
{
    const float2 jx = add2(sub2(sub2(add2(sub2(g[1], g[3]), g[5]), g[6]), g[7]), g[8]);
    const float2 jy = sub2(sub2(add2(add2(sub2(g[2], g[4]), g[5]), g[6]), g[7]), g[8]);
    float2 rr;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rr.x) : "f"(rho.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rr.y) : "f"(rho.y));
    const float2 k = mul2(f2(c.cmu), rr);
    const float2 usx = mul2(jx, k), usy = mul2(jy, k);
    const float2 A = fma2(f2(-1.5f), fma2(usx, usx, mul2(usy, usy)), f2(1.0f));
    const float2 r1 = mul2(f2(c.ow1), rho), r5 = mul2(f2(c.ow5), rho);
    const float2 om1 = f2(c.om1), p3 = f2(3.0f), m3 = f2(-3.0f), h45 = f2(4.5f);
    float2 e, p;
    e = usx;
    p = fma2(mul2(h45, e), e, A);
    fo[1] = fma2(om1, g[1], fma2(r1, fma2(p3, e, p), eta[1]));
    fo[3] = fma2(om1, g[3], fma2(r1, fma2(m3, e, p), eta[3]));
    e = usy;
    p = fma2(mul2(h45, e), e, A);
    fo[2] = fma2(om1, g[2], fma2(r1, fma2(p3, e, p), eta[2]));
    fo[4] = fma2(om1, g[4], fma2(r1, fma2(m3, e, p), eta[4]));
    e = add2(usx, usy);
    p = fma2(mul2(h45, e), e, A);
    fo[5] = fma2(om1, g[5], fma2(r5, fma2(p3, e, p), eta[5]));
    fo[7] = fma2(om1, g[7], fma2(r5, fma2(m3, e, p), eta[7]));
    e = sub2(usy, usx);
    p = fma2(mul2(h45, e), e, A);
    fo[6] = fma2(om1, g[6], fma2(r5, fma2(p3, e, p), eta[6]));
    fo[8] = fma2(om1, g[8], fma2(r5, fma2(m3, e, p), eta[8]));
    fo[0] = sub2(rho, add2(add2(add2(fo[1], fo[2]), add2(fo[3], fo[4])), add2(add2(fo[5], fo[6]), add2(fo[7], fo[8]))));
}

// relax_words<float, NOISE> for two nodes.
template <bool NOISE>
__device__ __forceinline__ void relax_pair(const float2 g[NQ], float2 rho, float2 fo[NQ], const u32x4 &wa,
                                           const u32x4 &wb, const Consts<float> &c)
{
    float2 eta[NQ];
    if constexpr (NOISE) {
        noise_eta_pair(eta, wa, wb, c);
    } else {
#pragma unroll
        for (int i = 0; i < NQ; ++i) eta[i] = f2(0.0f);
    }
    collide_pair(g, rho, fo, c, eta);
}

} // namespace lbm
