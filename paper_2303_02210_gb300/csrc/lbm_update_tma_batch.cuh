// TMA-staged fused update of a whole batch of simulations in one launch (FP32
// or 16-bit storage, walls in y, D2Q9): App. A steps 1, 2, 4-7 for every
// member, with step 3's divisions already added to the stored slots by the
// batched injection launch. The per-node arithmetic is k_update_tma's (and so
// k_update's, bit for bit); only the work distribution differs.
//
// Work. Every CTA first reads each member's step and window [y_r, y_hi) and
// forms, in shared memory, the exclusive prefix of the members' tile counts
// (128 x 2 tiles of their windows): the batch's tiles, member after member.
// The tiles are dealt in chunks of kTmaBatchChunk consecutive tiles, chunk j
// to CTA j mod G, so all members advance together. A CTA that moves on to
// another member fences that member's tensor map before its first copy
// through it (a map written to global memory by the host) and flushes its
// accumulators: with one tile per chunk, as the single-lattice kernel deals
// a lattice's tiles, a CTA changed member at nearly every tile (members of
// a few hundred tiles, a grid of 760 CTAs), and on the 256-member ensemble
// chunks of 2, 4 and 8 tiles took the step from 0.551 to 0.527, 0.516 and
// 0.513 ms. The producer (thread 0) looks up
// the member of each tile it issues (binary search in the prefix), copies its
// box through that member's tensor map (kept in global memory, one per
// population copy and member) and leaves the member and the tile's place in a
// per-stage record that the consumers read.
//
// Each member's constants (a 128-byte MemberConst block, built once per
// batch) travel with its tiles: the producer copies the block into the
// stage's record with an untiled bulk copy that completes on the same barrier
// as the tile's box, so the consumers find the box and the constants in
// shared memory together (per-tile global loads of them stalled this kernel
// on the L2's latency). The Philox round keys are built from the member's two
// key words. The mass and top-mass-row accumulators go to the member's
// scalars when the CTA moves on to another member and at the end (the
// negative fix's added mass only when some lane has any).
#pragma once

#include "lbm_update_tma.cuh"

namespace lbm {

// (TSTORE: an output tile [plane][2][128] more, for bulk tensor stores)
template <typename S, int STAGES, bool TSTORE = false>
constexpr size_t tma_batch_smem_bytes()
{
    return 128 + (size_t)STAGES * TmaGeom<S, 2>::STRIDE * sizeof(S) + (size_t)STAGES * sizeof(MemberConst) +
           (TSTORE ? (size_t)9 * 2 * TMA_TX * sizeof(S) : 0) + 16 * STAGES + (size_t)STAGES * 16 +
           (size_t)(kTmaBatchMaxSims + 1) * 4 + (size_t)kTmaBatchMaxSims * 4 * 4;
}

template <typename S>
struct TmaBatchCfg {
    // two stages for 16-bit storage too: on the 256-member ensemble in FP16,
    // 0.504 ms per step against 0.684 with four stages (and 0.517 with six
    // CTAs per SM of two stages, which spill)
    static constexpr int STAGES = 2, CTAS = kTmaBatchCtasPerSm;
    // the bulk-store form (FP32): one stage and six CTAs per SM, as the
    // single-lattice bulk-store form (latency-bound: more warps beat a
    // second stage)
    static constexpr int STAGES_ST = 1, CTAS_ST = kTmaBatchCtasPerSmStore;
};
static_assert(kTmaBatchCtasPerSmStore * (tma_batch_smem_bytes<float, 1, true>() + 1024) <= 228 * 1024,
              "the bulk-store form's CTAs per SM by shared memory");
static_assert(5 * (tma_batch_smem_bytes<float, 2>() + 1024) <= 228 * 1024, "five CTAs per SM");
static_assert(5 * (tma_batch_smem_bytes<__half, 2>() + 1024) <= 228 * 1024, "five CTAs per SM");

// Philox4x32-10 with the round keys formed as it goes (k + r x Weyl
// constant): the same values as philox4x32_10 with philox_key(k0, k1).
__device__ __forceinline__ u32x4 philox4x32_10_k(u32x4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c.z;
        c = u32x4{(uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// maps[4 m + b]: member m's copy b for loads ((kTmaBoxX + 8) x 4 x 9 boxes),
// maps[4 m + 2 + b] for bulk stores (TSTORE: kTmaBoxX x 2 x 9, cut at
// x = W - 1).
template <typename S, int STAGES, int CTAS, bool NOISE, bool TSTORE>
__global__ void __launch_bounds__(TmaGeom<S, 2>::NT, CTAS)
    k_update_tma_batch(const MemberConst *__restrict__ mc, const CUtensorMap *maps, int nsims)
{
    static_assert(!TSTORE || sizeof(S) == 4, "bulk tensor stores of 16-bit tiles would start off a 16-byte boundary");
    constexpr int TY = 2;
    using G = TmaGeom<S, TY>;
    constexpr int NT = G::NT, PLANE = G::PLANE;
    extern __shared__ __align__(128) float smem_f[];
    S *s_in = reinterpret_cast<S *>(smem_f + ((128u - (smem_u32(smem_f) & 127u)) & 127u) / 4u);
    MemberConst *s_mc = reinterpret_cast<MemberConst *>(s_in + STAGES * G::STRIDE); // per stage, 128-byte aligned
    S *s_out = reinterpret_cast<S *>(s_mc + STAGES);                                 // the output tile (TSTORE)
    uint64_t *full = reinterpret_cast<uint64_t *>(s_out + (TSTORE ? 9 * TY * TMA_TX : 0));
    uint64_t *empty = full + STAGES;
    int4 *s_tile = reinterpret_cast<int4 *>(empty + STAGES); // per stage: member, x0, y0, -
    int *s_pre = reinterpret_cast<int *>(s_tile + STAGES);    // nsims + 1 tile prefixes
    int *s_step = s_pre + kTmaBatchMaxSims + 1;
    int *s_yr = s_step + kTmaBatchMaxSims;
    int *s_yhi = s_yr + kTmaBatchMaxSims;
    int *s_ncx = s_yhi + kTmaBatchMaxSims; // column tiles
    __shared__ int s_abort;
    __shared__ int s_wsum[NT / 32];
    __shared__ unsigned s_fenced[4 * kTmaBatchMaxSims / 32]; // maps this CTA has made visible to the TMA unit
    __shared__ unsigned s_frz[kTmaBatchMaxSims / 32];        // members whose rear wall froze rows last step
    constexpr int K = (kTmaBatchMaxSims + NT - 1) / NT; // members per thread in the prologue

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int half = warp & 1, row = warp >> 1;
    if (tid < 4 * kTmaBatchMaxSims / 32) s_fenced[tid] = 0u;
    if (tid < kTmaBatchMaxSims / 32) s_frz[tid] = 0u;
    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], G::WARPS);
            s_tile[s] = make_int4(0, 0, 0, 0); // (read only by a consumer whose wait gave up)
        }
        fence_mbar_init();
    }
    // the members' steps and windows, and their tile counts
    int cnt[K];
    int mine = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int m = tid * K + j;
        cnt[j] = 0;
        const DevScalars *sc = m < nsims ? mc[m].sc : nullptr;
        if (m < nsims && !sc) s_step[m] = s_yr[m] = s_yhi[m] = s_ncx[m] = 0; // an empty slot: no tiles
        if (sc) {
            const int y_r = sc->y_r, y_hi = sc->y_hi;
            s_step[m] = (int)sc->step;
            s_yr[m] = y_r;
            s_yhi[m] = y_hi;
            const int ncx = (mc[m].W + TMA_TX - 1) / TMA_TX;
            s_ncx[m] = ncx;
            const int nrows = y_hi - y_r;
            cnt[j] = nrows > 0 ? ncx * ((nrows + TY - 1) / TY) : 0;
            if (sc->y_copy < y_r) atomicOr(&s_frz[m >> 5], 1u << (m & 31));
        }
        mine += cnt[j];
    }
    // exclusive prefix over the members
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    int before = incl - mine;
    for (int i = 0; i < warp; ++i) before += s_wsum[i];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int m = tid * K + j;
        if (m < nsims) s_pre[m] = before;
        before += cnt[j];
    }
    if (tid == NT - 1) s_pre[nsims] = before; // (the last thread's running sum: all tiles)
    __syncthreads();
    const int T = s_pre[nsims];
    const long long budget = kWaitBudget;

    // rows the rear walls have just frozen: bring the copies up to date
    for (int m = 0; m < nsims; ++m) {
        if (!((s_frz[m >> 5] >> (m & 31)) & 1u)) continue;
        const int y_copy = mc[m].sc->y_copy, y_r = s_yr[m];
        const int cur = s_step[m] & 1;
        const S *fin = (const S *)mc[m].f[cur];
        S *fout = (S *)mc[m].f[cur ^ 1];
        const long long P = mc[m].P, Wp = mc[m].Wp;
        const long long n = (long long)(y_r - y_copy) * Wp;
        for (long long k = (long long)blockIdx.x * NT + tid; k < n; k += (long long)gridDim.x * NT) {
            const long long o = (long long)y_copy * Wp + k - kXO;
#pragma unroll
            for (int i = 0; i < NQ; ++i) fout[i * P + o] = fin[i * P + o];
        }
    }

    const int Gd = (int)gridDim.x;
    // the batch's tiles dealt in chunks of C consecutive tiles: chunk j to
    // CTA j mod G (a CTA's tiles then change member, which costs a tensor-map
    // fence and an accumulator flush, C times less often)
    constexpr int C = kTmaBatchChunk;
    const int nchunks = (T + C - 1) / C;
    const int nmine = (int)blockIdx.x < nchunks ? (nchunks - 1 - (int)blockIdx.x) / Gd + 1 : 0;
    const int count = nmine > 0 ? (nmine - 1) * C + min(C, T - ((int)blockIdx.x + (nmine - 1) * Gd) * C) : 0;
    // the member of tile g: the last m with s_pre[m] <= g
    auto member_of = [&](int g) {
        int lo = 0, hi = nsims - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_pre[mid] <= g) lo = mid; else hi = mid - 1;
        }
        return lo;
    };
    // a map lives in global memory, written before the launch: make it
    // visible to the tensor-map proxy, once per map and CTA (thread 0)
    auto fence_map = [&](int mi) {
        if (!((s_fenced[mi >> 5] >> (mi & 31)) & 1u)) {
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)(maps + mi))
                         : "memory");
            s_fenced[mi >> 5] |= 1u << (mi & 31);
        }
    };
    int issued = 0;
    auto issue = [&]() {
        const int s = issued % STAGES;
        const int g = ((int)blockIdx.x + (issued / C) * Gd) * C + issued % C;
        const int m = member_of(g);
        const int lt = g - s_pre[m];
        const int ncx = s_ncx[m];
        const int tx = lt % ncx, ty = lt / ncx;
        const int x0 = tx * TMA_TX, y0 = s_yr[m] + ty * TY;
        s_tile[s] = make_int4(m, x0, y0, 0);
        const int mi = 4 * m + (s_step[m] & 1);
        const CUtensorMap *tm = maps + mi;
        fence_map(mi);
        mbar_arrive_expect_tx(&full[s], G::BYTES + (uint32_t)sizeof(MemberConst));
        tma_load_3d(s_in + s * G::STRIDE, tm, x0 - 4 + kXO, y0 - 1, 0, &full[s]);
        bulk_load(&s_mc[s], &mc[m], (uint32_t)sizeof(MemberConst), &full[s]);
        ++issued;
    };
    if (tid == 0)
        while (issued < STAGES && issued < count) issue();

    const int cl = 64 * half + 2 * lane;
    long long mass = 0;
    int maxrow = -1;
    float clip = 0.0f;
    int acc_m = -1;             // the member the accumulators belong to
    DevScalars *acc_sc = nullptr;
    bool dead = false;
    // the accumulators go to member acc_m (warp sums, one atomic per warp)
    auto flush = [&]() {
        const long long ms = warp_sum_ll(mass);
        const int mr = warp_max_i(maxrow);
        const bool any_clip = __any_sync(0xffffffffu, clip != 0.0f);
        const double cd = any_clip ? warp_sum_d((double)clip) : 0.0;
        if (lane == 0 && acc_sc) {
            if (ms != 0) atomicAdd(&acc_sc->mass_accum, (unsigned long long)ms);
            if (mr >= 0) atomicMax(&acc_sc->maxmass_accum, mr);
            if (cd != 0.0) atomicAdd(&acc_sc->clip_mass, cd);
        }
        mass = 0;
        maxrow = -1;
        clip = 0.0f;
    };

    for (int k = 0; k < count; ++k) {
        const int s = k % STAGES;
        const uint32_t parity = (uint32_t)((k / STAGES) & 1);
        S *stage = s_in + s * G::STRIDE;
        if (!dead && !mbar_wait_bounded(&full[s], parity, budget)) {
            dead = true;
            atomicOr(&s_abort, 1);
        }
        const int4 ti = s_tile[s];
        const int m = min(max(ti.x, 0), nsims - 1), x0 = ti.y, y0 = ti.z;
        const MemberConst &c = s_mc[s];
        if (m != acc_m) { // uniform across the CTA
            flush();
            acc_m = m;
            acc_sc = c.sc;
        }
        const Pop<S> pc(c.pop_shift);
        const int W = c.W, H = c.H;
        const int y_r = s_yr[m], y_hi = s_yhi[m];
        const uint32_t t = (uint32_t)s_step[m];
        const int y = y0 + row;
        const bool active = y < y_hi;
        float2 g2[NQ];
        // (the record's other fields, read now: the stage is released below)
        const long long P = c.P;
        const int Wp = c.Wp, MW = c.MW;
        S *fout = (S *)c.f[(t & 1u) ^ 1u];
        uint32_t *mask = c.mask;
        const Consts<float> cf{0.0f, c.cmu, c.om1, 0.0f, c.ow1, c.ow5, c.two_sigma};
        const float rho_c = c.rho_c;
        const int negfix = c.negfix;
        const uint32_t key0 = c.key0, key1 = c.key1, sim = c.sim;
        if (active) {
            const S *b = stage + (row + 1) * TMA_LX + cl + 4;
            const bool rear = y - 1 < y_r, top = y + 1 >= H;
            if (!rear && !top)
                pull2p<S, PLANE, false, false>(b, g2, pc);
            else if (!top)
                pull2p<S, PLANE, true, false>(b, g2, pc);
            else if (!rear)
                pull2p<S, PLANE, false, true>(b, g2, pc);
            else
                pull2p<S, PLANE, true, true>(b, g2, pc);
        }
        // the stage (box and record) may be refilled once every warp has its
        // values
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (tid == 0 && issued < count) {
            if (!dead && !mbar_wait_bounded(&empty[s], parity, budget)) {
                dead = true;
                atomicOr(&s_abort, 1);
            }
            if (!dead) issue();
        }
        float2 res[NQ]; // this thread's two nodes' results (TSTORE)
        if (active) {
            const int x = x0 + cl;
            const bool oka = x < W, okb = x + 1 < W;
            const float2 rho2 = rho_pair(g2);
            const float rhoa = rho2.x, rhob = rho2.y;
            const bool occa = oka && rhoa >= rho_c, occb = okb && rhob >= rho_c;
            S *o = fout + (long long)y * Wp + x;
            if (__all_sync(0xffffffffu, occa && occb)) {
                const uint32_t n = (uint32_t)(y * W + x);
                const u32x4 wa = NOISE ? philox4x32_10_k(u32x4{n, t, STREAM_NOISE, sim}, key0, key1)
                                       : u32x4{0u, 0u, 0u, 0u};
                const u32x4 wb = NOISE ? philox4x32_10_k(u32x4{n + 1u, t, STREAM_NOISE, sim}, key0, key1)
                                       : u32x4{0u, 0u, 0u, 0u};
                float2 f2o[NQ];
                relax_pair<NOISE>(g2, rho2, f2o, wa, wb, cf);
                float mn = fminf(f2o[0].x, f2o[0].y);
#pragma unroll
                for (int i = 1; i < NQ; ++i) mn = fminf(mn, fminf(f2o[i].x, f2o[i].y));
                float adda = 0.0f, addb = 0.0f;
                if (__any_sync(0xffffffffu, mn < 0.0f)) {
                    float fa[NQ], fb[NQ];
#pragma unroll
                    for (int i = 0; i < NQ; ++i) {
                        fa[i] = f2o[i].x;
                        fb[i] = f2o[i].y;
                    }
                    adda = fix_negative<float>(fa, negfix);
                    addb = fix_negative<float>(fb, negfix);
#pragma unroll
                    for (int i = 0; i < NQ; ++i) f2o[i] = make_float2(fa[i], fb[i]);
                    clip += adda + addb;
                }
                if ((lane & 15) == 0) mask[(long long)y * MW + (x0 >> 5) + 2 * half + (lane >> 4)] = 0xffffffffu;
                float2 m2 = f2(0.0f);
                if constexpr (TSTORE) {
#pragma unroll
                    for (int i = 0; i < NQ; ++i) res[i] = f2o[i];
                } else {
                    store_pair<S>(o, P, f2o, pc, m2);
                }
                const int xw = x0 + 64 * half;
                if (xw == 0 || xw + 63 == W - 1) {
                    if (x == 0) {
#pragma unroll
                        for (int i = 0; i < NQ; ++i) o[i * P + W] = pc.st(f2o[i].x, i);
                    }
                    if (x + 1 == W - 1) {
#pragma unroll
                        for (int i = 0; i < NQ; ++i) o[i * P + 1 - W] = pc.st(f2o[i].y, i);
                    }
                }
                const float roa = Pop<S>::kShifted ? m2.x : rhoa + adda;
                const float rob = Pop<S>::kShifted ? m2.y : rhob + addb;
                mass += fix24<float>(roa) + fix24<float>(rob);
                if (roa != 0.0f || rob != 0.0f) maxrow = y;
            } else {
                float ga[NQ], gb[NQ];
#pragma unroll
                for (int i = 0; i < NQ; ++i) {
                    ga[i] = g2[i].x;
                    gb[i] = g2[i].y;
                }
                u32x4 wa{0u, 0u, 0u, 0u}, wb{0u, 0u, 0u, 0u};
                if (NOISE && (occa || occb)) {
                    const uint32_t n = (uint32_t)(y * W + x);
                    wa = philox4x32_10_k(u32x4{n, t, STREAM_NOISE, sim}, key0, key1);
                    wb = philox4x32_10_k(u32x4{n + 1u, t, STREAM_NOISE, sim}, key0, key1);
                }
                float fa[NQ], fb[NQ];
                const float adda = update_node<NOISE>(ga, rhoa, occa, fa, wa, cf, negfix);
                const float addb = update_node<NOISE>(gb, rhob, occb, fb, wb, cf, negfix);
                unsigned v = ((unsigned)occa | ((unsigned)occb << 1)) << (2 * (lane & 15));
                v |= __shfl_xor_sync(0xffffffffu, v, 1);
                v |= __shfl_xor_sync(0xffffffffu, v, 2);
                v |= __shfl_xor_sync(0xffffffffu, v, 4);
                v |= __shfl_xor_sync(0xffffffffu, v, 8);
                const int word = (x0 >> 5) + 2 * half + (lane >> 4);
                if ((lane & 15) == 0 && word < MW) mask[(long long)y * MW + word] = v;
                float ma = 0.0f, mb = 0.0f;
                if constexpr (TSTORE) {
#pragma unroll
                    for (int i = 0; i < NQ; ++i) res[i] = make_float2(fa[i], fb[i]);
                } else {
                    if (oka) store_nodes<S>(o, P, fa, fb, okb, pc, ma, mb);
                }
                if (x == 0) {
#pragma unroll
                    for (int i = 0; i < NQ; ++i) o[i * P + W] = pc.st(fa[i], i);
                }
                if (x == W - 1) {
#pragma unroll
                    for (int i = 0; i < NQ; ++i) o[i * P - W] = pc.st(fa[i], i);
                }
                if (x + 1 == W - 1) {
#pragma unroll
                    for (int i = 0; i < NQ; ++i) o[i * P + 1 - W] = pc.st(fb[i], i);
                }
                if (oka) {
                    clip += adda;
                    const float ro = Pop<S>::kShifted ? ma : rhoa + adda;
                    mass += fix24<float>(ro);
                    if (ro != 0.0f) maxrow = y;
                }
                if (okb) {
                    clip += addb;
                    const float ro = Pop<S>::kShifted ? mb : rhob + addb;
                    mass += fix24<float>(ro);
                    if (ro != 0.0f) maxrow = y;
                }
            }
        }
        if constexpr (TSTORE) {
            // the previous tile's store must have read the output tile
            if (tid == 0) bulk_wait_read<0>();
            __syncthreads();
            // rows past the window get zeros, which they hold anyway; columns
            // from x = W on are cut by the store's tensor map
            S *ot = s_out + row * TMA_TX + cl;
#pragma unroll
            for (int i = 0; i < NQ; ++i)
                *reinterpret_cast<float2 *>(ot + i * TY * TMA_TX) = active ? res[i] : f2(0.0f);
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                const int mi = 4 * m + 2 + (int)((t & 1u) ^ 1u);
                fence_map(mi);
                tma_store_3d(maps + mi, x0 + kXO, y0, 0, s_out);
                bulk_commit();
            }
        }
    }
    if (TSTORE && tid == 0) bulk_wait_all();
    if (tid == 0 && s_abort) {
        for (int m = 0; m < nsims; ++m) atomicOr(&mc[m].sc->status, ST_TIMEOUT);
        for (int k = issued - STAGES > 0 ? issued - STAGES : 0; k < issued; ++k)
            mbar_wait_bounded(&full[k % STAGES], (uint32_t)((k / STAGES) & 1), kWaitBudget);
    }
    flush();
}

template <typename S, bool NOISE, bool TSTORE>
cudaError_t launch_update_tma_batch_n(const MemberConst *mc, const CUtensorMap *maps, int n, int grid,
                                      cudaStream_t s)
{
    using C = TmaBatchCfg<S>;
    constexpr int CTAS = TSTORE ? C::CTAS_ST : C::CTAS;
    constexpr int ST = TSTORE ? C::STAGES_ST : C::STAGES;
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !attr[dev]) {
        e = cudaFuncSetAttribute(k_update_tma_batch<S, ST, CTAS, NOISE, TSTORE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tma_batch_smem_bytes<S, ST, TSTORE>());
        if (e != cudaSuccess) return e;
        if (dev < 64) attr[dev] = true;
    }
    k_update_tma_batch<S, ST, CTAS, NOISE, TSTORE>
        <<<grid, TmaGeom<S, 2>::NT, tma_batch_smem_bytes<S, ST, TSTORE>(), s>>>(mc, maps, n);
    return cudaGetLastError();
}

// noise: whether any member has sigma != 0 (a member with sigma = 0 then
// draws noise blocks it does not need: its eta comes out +0 exactly, the
// value the noise-free form adds, so the results are the same bit for bit);
// tstore: the members' results leave by bulk tensor stores (FP32, every
// width a multiple of 4; grid at most CTAS_ST per SM)
template <typename S>
cudaError_t launch_update_tma_batch(const SimDev *, const MemberConst *mc, const CUtensorMap *maps, int n,
                                    int noise, int tstore, int grid, cudaStream_t s)
{
    if constexpr (sizeof(S) == 4)
        if (tstore)
            return noise ? launch_update_tma_batch_n<S, true, true>(mc, maps, n, grid, s)
                         : launch_update_tma_batch_n<S, false, true>(mc, maps, n, grid, s);
    return noise ? launch_update_tma_batch_n<S, true, false>(mc, maps, n, grid, s)
                 : launch_update_tma_batch_n<S, false, false>(mc, maps, n, grid, s);
}

} // namespace lbm
