// TMA-staged fused update on the triangular D2Q7 lattice (FP32 storage,
// walls in y): App. A steps 1, 2 and 4-7 with the per-node arithmetic of
// update7_body (the same functions, in the same order, so the two kernels
// agree bit for bit), and the data movement of k_update_tma.
//
// Each CTA (persistent, CTAS per SM) walks tiles of 128 columns x TY rows of
// the active window, dealt round-robin over the grid. A tile's pre-stream
// populations arrive in shared memory as one 3-D bulk tensor copy of box
// 136 x (TY + 2) x 7 floats (the tile, four stored columns on each side,
// which hold the ghost columns -1 and W, one row below and one above, all
// seven planes); STAGES boxes in flight per CTA, full/empty mbarriers, and
// step 3's divisions added to the staged pre-stream slots from the CTA's
// record bucket (division_record7), all as in k_update_tma.
//
// Streaming on the triangular lattice (Sec. II; odd rows sit half a spacing
// to the right): a node (x, y) pulls q = 1 from (x - 1, y), q = 4 from
// (x + 1, y), q = 2 from (x - 1 + par, y - 1), q = 3 from (x + par, y - 1),
// q = 5 from (x + par, y + 1) and q = 6 from (x - 1 + par, y + 1), par = y & 1.
// Each lane takes two adjacent nodes of one row, so par is warp-uniform: the
// planes whose source column offset is 0 are one paired shared load for both
// nodes, the others two scalar loads.
#pragma once

#include "lbm_d2q7.cuh"
#include "lbm_tma.cuh"
#include "lbm_update_tma.cuh"

namespace lbm {

template <int TY>
struct Tma7Geom {
    static constexpr int NT = 64 * TY; // threads: two warps per tile row
    static constexpr int LY = TY + 2;
    static constexpr int PLANE = LY * TMA_LX;                      // floats per staged plane
    static constexpr int IN_ELEMS = NQ7 * PLANE;                   // one box
    static constexpr int STRIDE = (IN_ELEMS * 4 + 127) / 128 * 128 / 4; // stage pitch (floats)
    static constexpr uint32_t BYTES = (uint32_t)IN_ELEMS * 4u;     // one box copy delivers
};

template <int TY, int STAGES>
constexpr size_t tma7_smem_bytes()
{
    return 128 + (size_t)STAGES * Tma7Geom<TY>::STRIDE * 4 + 16 * STAGES + (size_t)TMA_EV_CAP * 16 +
           TMA_KFLAG_WORDS * 4;
}

// The one configuration: tiles of two rows, 128 threads, two staged boxes per
// CTA, five CTAs per SM (the D2Q9 kernel's variant 0 on 7-plane boxes).
constexpr int TMA7_TY = 2, TMA7_STAGES = 2, TMA7_CTAS = 5;
static_assert(TMA7_CTAS * (tma7_smem_bytes<TMA7_TY, TMA7_STAGES>() + 1024) <= 228 * 1024,
              "five CTAs per SM by shared memory");

// Plane q of a node pair from the staged box: `p` points at the source of
// the first node; a paired load if the source column offset is even (the
// pair then starts on a pair boundary), else two scalar loads.
template <bool ALIGNED>
__device__ __forceinline__ void ld7(const float *p, float &a, float &b)
{
    if constexpr (ALIGNED) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        a = v.x;
        b = v.y;
    } else {
        a = p[0];
        b = p[1];
    }
}

// The populations two adjacent nodes of a row of parity ODD pull: `b` points
// at the first node's staged plane-0 value (on a pair boundary). Across the
// rear (REAR) or top (TOP) wall a node takes its own opposite population
// (half-way bounce-back, q <-> q + 3).
template <int PLANE, bool ODD, bool REAR, bool TOP>
__device__ __forceinline__ void pull7(const float *b, float ga[NQ7], float gb[NQ7])
{
    ld7<true>(b, ga[0], gb[0]);
    ld7<false>(b + PLANE - 1, ga[1], gb[1]);
    ld7<false>(b + 4 * PLANE + 1, ga[4], gb[4]);
    if (REAR) {
        ld7<true>(b + 5 * PLANE, ga[2], gb[2]);
        ld7<true>(b + 6 * PLANE, ga[3], gb[3]);
    } else if (ODD) {
        ld7<true>(b + 2 * PLANE - TMA_LX, ga[2], gb[2]);
        ld7<false>(b + 3 * PLANE - TMA_LX + 1, ga[3], gb[3]);
    } else {
        ld7<false>(b + 2 * PLANE - TMA_LX - 1, ga[2], gb[2]);
        ld7<true>(b + 3 * PLANE - TMA_LX, ga[3], gb[3]);
    }
    if (TOP) {
        ld7<true>(b + 2 * PLANE, ga[5], gb[5]);
        ld7<true>(b + 3 * PLANE, ga[6], gb[6]);
    } else if (ODD) {
        ld7<false>(b + 5 * PLANE + TMA_LX + 1, ga[5], gb[5]);
        ld7<true>(b + 6 * PLANE + TMA_LX, ga[6], gb[6]);
    } else {
        ld7<true>(b + 5 * PLANE + TMA_LX, ga[5], gb[5]);
        ld7<false>(b + 6 * PLANE + TMA_LX - 1, ga[6], gb[6]);
    }
}

template <int PLANE, bool ODD>
__device__ __forceinline__ void pull7_walls(const float *b, bool rear, bool top, float ga[NQ7], float gb[NQ7])
{
    if (!rear && !top)
        pull7<PLANE, ODD, false, false>(b, ga, gb);
    else if (!top)
        pull7<PLANE, ODD, true, false>(b, ga, gb);
    else if (!rear)
        pull7<PLANE, ODD, false, true>(b, ga, gb);
    else
        pull7<PLANE, ODD, true, true>(b, ga, gb);
}

// One node as update7_body computes it: relaxation with the Eq. 4 noise (or
// the reversal below rho_c), the negative fix; returns the mass the fix added.
template <bool NOISE>
__device__ __forceinline__ float update_node7(const float g[NQ7], float rho, bool occ, float fo[NQ7], const u32x4 &w,
                                              const Consts<float> &cf, int negfix)
{
    if (occ) {
        if (NOISE) {
            float eta[NQ7];
            noise_eta7<float>(eta, w, cf);
            collide7<float>(g, rho, fo, cf, eta);
        } else {
            collide7<float>(g, rho, fo, cf, nullptr);
        }
        return fix_negative7<float>(fo, negfix);
    }
#pragma unroll
    for (int i = 0; i < NQ7; ++i) fo[i] = g[opp7(i)];
    return 0.0f;
}

// Stores a node pair's results (columns x, x + 1 at `o`: paired stores), or
// the first node's alone if !both.
__device__ __forceinline__ void store_nodes7(float *o, long long P, const float fa[NQ7], const float fb[NQ7], bool both)
{
#pragma unroll
    for (int i = 0; i < NQ7; ++i) {
        if (both)
            *reinterpret_cast<float2 *>(o + i * P) = make_float2(fa[i], fb[i]);
        else
            o[i * P] = fa[i];
    }
}

template <int TY, int STAGES, int CTAS, bool NOISE>
__global__ void __launch_bounds__(Tma7Geom<TY>::NT, CTAS)
    k_update7_tma(SimDev d, const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1)
{
    using G = Tma7Geom<TY>;
    constexpr int NT = G::NT, PLANE = G::PLANE, WARPS = NT / 32;
    extern __shared__ __align__(128) float smem_f[];
    // stages on a 128-byte boundary (offset from the array itself)
    float *s_in = smem_f + ((128u - (smem_u32(smem_f) & 127u)) & 127u) / 4u;
    uint64_t *full = reinterpret_cast<uint64_t *>(s_in + STAGES * G::STRIDE);
    uint64_t *empty = full + STAGES;
    // divisions of this CTA's tiles: local tile index, two staged offsets, amount
    int *ev_k = reinterpret_cast<int *>(empty + STAGES);
    int *ev_off = ev_k + TMA_EV_CAP;
    float *ev_add = reinterpret_cast<float *>(ev_off + 2 * TMA_EV_CAP);
    unsigned *kflag = reinterpret_cast<unsigned *>(ev_add + TMA_EV_CAP); // tiles with divisions
    __shared__ int s_abort, s_nev;

    const int W = d.W, H = d.H, Wp = d.Wp;
    const long long P = d.P;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int half = warp & 1, row = warp >> 1; // column half and row of the tile

    // prologue, which may overlap the end of the kernel before (programmatic
    // dependent launch): barriers and tensor maps
    if (tid == 0) {
        s_abort = 0;
        s_nev = 0;
        prefetch_tensormap(&tm0);
        prefetch_tensormap(&tm1);
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], WARPS);
        }
        fence_mbar_init();
    }
    if (tid < TMA_KFLAG_WORDS) kflag[tid] = 0u;
    __syncthreads();
    grid_dependency_wait();
    const uint32_t t = (uint32_t)d.sc->step;
    // bounded waits: the budget (a failure-detection test shortens it and may
    // withhold the bulk copies, so that the first wait of every thread runs out)
    const long long budget = d.sc->wait_budget > 0 ? d.sc->wait_budget : kWaitBudget;
    const bool withhold = (d.sc->wait_test & WAIT_TEST_COPIES) != 0;
    const int cur = (int)(t & 1u);
    const CUtensorMap *tm = cur ? &tm1 : &tm0;
    const float *__restrict__ fin = (const float *)d.f[cur];
    float *__restrict__ fout = (float *)d.f[cur ^ 1];
    const int y_r = d.sc->y_r, y_copy = d.sc->y_copy, y_hi = d.sc->y_hi;

    // rows the rear wall has just frozen: bring this copy up to date (whole
    // stored rows, ghosts included)
    if (y_copy < y_r) {
        const long long n = (long long)(y_r - y_copy) * Wp;
        for (long long k = (long long)blockIdx.x * NT + tid; k < n; k += (long long)gridDim.x * NT) {
            const long long o = (long long)y_copy * Wp + k - kXO;
#pragma unroll
            for (int i = 0; i < NQ7; ++i) fout[i * P + o] = fin[i * P + o];
        }
    }

    const int ncx = (W + TMA_TX - 1) / TMA_TX;
    const int nrows = y_hi - y_r;
    const int nty = nrows > 0 ? (nrows + TY - 1) / TY : 0;
    const int ntiles = ncx * nty;
    const int Gd = (int)gridDim.x;
    const int count = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / Gd + 1 : 0;
    // tile k of this CTA is blockIdx.x + k Gd; its (tx, ty) advance by (Gd % ncx, Gd / ncx)
    const int dtx = Gd % ncx, dty = Gd / ncx;
    // producer state (thread 0): next tile to load and copies issued
    int itx = (int)blockIdx.x % ncx, ity = (int)blockIdx.x / ncx, issued = 0;
    auto issue = [&]() {
        const int s = issued % STAGES;
        mbar_arrive_expect_tx(&full[s], G::BYTES);
        tma_load_3d(s_in + s * G::STRIDE, tm, itx * TMA_TX - 4 + kXO, y_r + ity * TY - 1, 0, &full[s]);
        ++issued;
        itx += dtx;
        ity += dty;
        if (itx >= ncx) {
            itx -= ncx;
            ++ity;
        }
    };
    // the first tiles' copies run while the divisions are sorted out below
    if (tid == 0 && !withhold)
        while (issued < STAGES && issued < count) issue();

    // App. A step 3 for this CTA, as in k_update_tma: the records of its
    // bucket (all records if the bucket overflowed)
    const int nev_all = d.inject_in_update ? d.sc->rec_n : 0;
    auto amount = [&](int e) {
        return (float)((double)d.ev_count[(size_t)(t & 1u) * (size_t)d.ns_max + (size_t)e] * d.half_cell);
    };
    const int mine = nev_all > 0 ? d.bucket_cnt[blockIdx.x] : 0;
    if (mine <= TMA_EV_CAP) { // (the bucket holds kBucketCap >= TMA_EV_CAP records)
        for (int j = tid; j < mine; j += NT) {
            const int e = d.bucket[blockIdx.x * kBucketCap + j];
            const int k = d.rec_k[e];
            ev_k[j] = k;
            ev_off[2 * j] = d.rec_off[2 * e];
            ev_off[2 * j + 1] = d.rec_off[2 * e + 1];
            ev_add[j] = amount(e);
            if (k < 32 * TMA_KFLAG_WORDS) atomicOr(&kflag[k >> 5], 1u << (k & 31));
        }
        if (tid == 0) s_nev = mine;
    } else {
        for (int e = tid; e < nev_all; e += NT) {
            if (d.rec_owner[e] != (int)blockIdx.x) continue;
            const int at = atomicAdd(&s_nev, 1);
            const int k = d.rec_k[e];
            if (at < TMA_EV_CAP) {
                ev_k[at] = k;
                ev_off[2 * at] = d.rec_off[2 * e];
                ev_off[2 * at + 1] = d.rec_off[2 * e + 1];
                ev_add[at] = amount(e);
            }
            if (k < 32 * TMA_KFLAG_WORDS) atomicOr(&kflag[k >> 5], 1u << (k & 31));
        }
    }
    __syncthreads();
    const int nev = s_nev;                     // divisions of this CTA
    const bool ev_overflow = nev > TMA_EV_CAP; // then scan the global list per tile

    const Consts<float> cf = make_consts<float>(d);
    const float rho_c = d.f_rho_c;
    const int negfix = d.negfix;
    const int cl = 64 * half + 2 * lane; // this thread's first column in the tile
    long long mass = 0;
    int maxrow = -1;
    float clip = 0.0f;
    bool dead = false; // a wait of this thread gave up: no more waits, same barriers
    int tx = (int)blockIdx.x % ncx, ty = (int)blockIdx.x / ncx;

    for (int k = 0; k < count; ++k) {
        const int s = k % STAGES;
        const uint32_t parity = (uint32_t)((k / STAGES) & 1);
        const int x0 = tx * TMA_TX, y0 = y_r + ty * TY;
        float *stage = s_in + s * G::STRIDE;
        if (!dead && !mbar_wait_bounded(&full[s], parity, budget)) {
            dead = true;
            atomicOr(&s_abort, 1);
        }
        // divisions of this tile, added to the staged pre-stream slots
        // (distinct records never share a slot)
        const bool has_ev =
            nev > 0 && (ev_overflow || k >= 32 * TMA_KFLAG_WORDS || ((kflag[k >> 5] >> (k & 31)) & 1u));
        if (has_ev) { // uniform across the CTA
            if (!ev_overflow) {
                for (int i = tid; i < nev; i += NT)
                    if (ev_k[i] == k) {
                        stage[ev_off[2 * i]] = stage[ev_off[2 * i]] + ev_add[i];
                        stage[ev_off[2 * i + 1]] = stage[ev_off[2 * i + 1]] + ev_add[i];
                    }
            } else {
                for (int e = tid; e < nev_all; e += NT)
                    if (d.rec_owner[e] == (int)blockIdx.x && d.rec_k[e] == k) {
                        const float a = amount(e);
                        stage[d.rec_off[2 * e]] = stage[d.rec_off[2 * e]] + a;
                        stage[d.rec_off[2 * e + 1]] = stage[d.rec_off[2 * e + 1]] + a;
                    }
            }
            fence_proxy_async_smem(); // before a later bulk copy overwrites them
            __syncthreads();
        }
        // the pulled populations of this thread's two nodes (rows past the
        // active window hold no mass and are skipped; warp-uniform)
        const int y = y0 + row;
        const bool active = y < y_hi;
        float ga[NQ7], gb[NQ7];
        if (active) {
            const float *b = stage + (row + 1) * TMA_LX + cl + 4;
            const bool rear = y - 1 < y_r, top = y + 1 >= H; // half-way bounce-back walls
            if (y & 1)
                pull7_walls<PLANE, true>(b, rear, top, ga, gb);
            else
                pull7_walls<PLANE, false>(b, rear, top, ga, gb);
        }
        // the stage may be refilled (by the async proxy) once every warp has
        // arrived: order this thread's shared-memory reads before that
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (tid == 0 && issued < count && !withhold) {
            if (!dead && !mbar_wait_bounded(&empty[s], parity, budget)) {
                dead = true;
                atomicOr(&s_abort, 1);
            }
            if (!dead) issue();
        }
        if (active) {
            const int x = x0 + cl;
            const bool oka = x < W, okb = x + 1 < W;
            float rhoa = ga[0], rhob = gb[0];
#pragma unroll
            for (int i = 1; i < NQ7; ++i) {
                rhoa = rhoa + ga[i];
                rhob = rhob + gb[i];
            }
            const bool occa = oka && rhoa >= rho_c, occb = okb && rhob >= rho_c;
            float *o = fout + (long long)y * Wp + x;
            if (__all_sync(0xffffffffu, occa && occb)) {
                // the bulk: all 64 nodes of the warp's segment are occupied
                // (and inside the lattice): no per-node branches, one full
                // mask word per 16 lanes, the fix only where a value went
                // negative (it leaves non-negative nodes as they are)
                const uint32_t n = (uint32_t)(y * W + x);
                float fa[NQ7], fb[NQ7];
                if (NOISE) {
                    float eta[NQ7];
                    noise_eta7<float>(eta, philox4x32_10(u32x4{n, t, STREAM_NOISE, d.sim}, d.pk), cf);
                    collide7<float>(ga, rhoa, fa, cf, eta);
                    noise_eta7<float>(eta, philox4x32_10(u32x4{n + 1u, t, STREAM_NOISE, d.sim}, d.pk), cf);
                    collide7<float>(gb, rhob, fb, cf, eta);
                } else {
                    collide7<float>(ga, rhoa, fa, cf, nullptr);
                    collide7<float>(gb, rhob, fb, cf, nullptr);
                }
                float mn = fminf(fa[0], fb[0]);
#pragma unroll
                for (int i = 1; i < NQ7; ++i) mn = fminf(mn, fminf(fa[i], fb[i]));
                float adda = 0.0f, addb = 0.0f;
                if (__any_sync(0xffffffffu, mn < 0.0f)) {
                    adda = fix_negative7<float>(fa, negfix);
                    addb = fix_negative7<float>(fb, negfix);
                    clip += adda;
                    clip += addb;
                }
                if ((lane & 15) == 0) d.mask[(long long)y * d.MW + (x0 >> 5) + 2 * half + (lane >> 4)] = 0xffffffffu;
                store_nodes7(o, P, fa, fb, true);
                const int xw = x0 + 64 * half; // first column of the warp
                if (xw == 0 || xw + 63 == W - 1) { // a warp at the lattice edge: ghost copies
                    if (x == 0) {
#pragma unroll
                        for (int i = 0; i < NQ7; ++i) o[i * P + W] = fa[i];
                    }
                    if (x + 1 == W - 1) {
#pragma unroll
                        for (int i = 0; i < NQ7; ++i) o[i * P + 1 - W] = fb[i];
                    }
                }
                const float roa = rhoa + adda, rob = rhob + addb;
                mass += fix24<float>(roa) + fix24<float>(rob);
                if (roa != 0.0f || rob != 0.0f) maxrow = y;
            } else {
                u32x4 wa{0u, 0u, 0u, 0u}, wb{0u, 0u, 0u, 0u};
                if (NOISE && (occa || occb)) {
                    const uint32_t n = (uint32_t)(y * W + x);
                    wa = philox4x32_10(u32x4{n, t, STREAM_NOISE, d.sim}, d.pk);
                    wb = philox4x32_10(u32x4{n + 1u, t, STREAM_NOISE, d.sim}, d.pk);
                }
                float fa[NQ7], fb[NQ7];
                const float adda = update_node7<NOISE>(ga, rhoa, occa, fa, wa, cf, negfix);
                const float addb = update_node7<NOISE>(gb, rhob, occb, fb, wb, cf, negfix);
                // occupancy bits: lanes 0-15 hold one 32-column word, lanes 16-31 the next
                unsigned v = ((unsigned)occa | ((unsigned)occb << 1)) << (2 * (lane & 15));
                v |= __shfl_xor_sync(0xffffffffu, v, 1);
                v |= __shfl_xor_sync(0xffffffffu, v, 2);
                v |= __shfl_xor_sync(0xffffffffu, v, 4);
                v |= __shfl_xor_sync(0xffffffffu, v, 8);
                const int word = (x0 >> 5) + 2 * half + (lane >> 4);
                if ((lane & 15) == 0 && word < d.MW) d.mask[(long long)y * d.MW + word] = v;
                // (odd W: the last column alone, x = W is the ghost)
                if (oka) store_nodes7(o, P, fa, fb, okb);
                // ghost copies of the edge columns for the next step's boxes
                if (x == 0) {
#pragma unroll
                    for (int i = 0; i < NQ7; ++i) o[i * P + W] = fa[i];
                }
                if (x == W - 1) {
#pragma unroll
                    for (int i = 0; i < NQ7; ++i) o[i * P - W] = fa[i];
                }
                if (x + 1 == W - 1) {
#pragma unroll
                    for (int i = 0; i < NQ7; ++i) o[i * P + 1 - W] = fb[i];
                }
                // the node's mass: rho plus what the fix added (as update7_body)
                if (oka) {
                    clip += adda;
                    const float ro = rhoa + adda;
                    mass += fix24<float>(ro);
                    if (ro != 0.0f) maxrow = y;
                }
                if (okb) {
                    clip += addb;
                    const float ro = rhob + addb;
                    mass += fix24<float>(ro);
                    if (ro != 0.0f) maxrow = y;
                }
            }
        }
        tx += dtx;
        ty += dty;
        if (tx >= ncx) {
            tx -= ncx;
            ++ty;
        }
    }
    if (tid == 0 && s_abort) {
        atomicOr(&d.sc->status, ST_TIMEOUT);
        // let the copies still in flight land before the CTA exits
        for (int k = issued - STAGES > 0 ? issued - STAGES : 0; k < issued; ++k)
            mbar_wait_bounded(&full[k % STAGES], (uint32_t)((k / STAGES) & 1), kWaitBudget);
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

// The kernel's shared-memory opt-in (once per device).
template <bool NOISE>
cudaError_t prepare_update7_tma()
{
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !attr[dev]) {
        e = cudaFuncSetAttribute(k_update7_tma<TMA7_TY, TMA7_STAGES, TMA7_CTAS, NOISE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tma7_smem_bytes<TMA7_TY, TMA7_STAGES>());
        if (e != cudaSuccess) return e;
        if (dev < 64) attr[dev] = true;
    }
    return cudaSuccess;
}

inline cudaError_t prepare_update7_tma_any(const SimDev &d, int)
{
    return d.noise_on ? prepare_update7_tma<true>() : prepare_update7_tma<false>();
}

// maps[b] loads from population copy b (boxes of 136 x 4 x 7). Launched as a
// programmatic dependent of the kernel before it when pdl is set.
template <bool NOISE>
cudaError_t launch_update7_tma(const SimDev &d, const CUtensorMap *maps, bool pdl, cudaStream_t s)
{
    cudaError_t e = prepare_update7_tma<NOISE>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)d.upd_ctas); // at most TMA7_CTAS per SM
    cfg.blockDim = dim3(Tma7Geom<TMA7_TY>::NT);
    cfg.dynamicSmemBytes = tma7_smem_bytes<TMA7_TY, TMA7_STAGES>();
    cfg.stream = s;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    la[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = la;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_update7_tma<TMA7_TY, TMA7_STAGES, TMA7_CTAS, NOISE>, d, maps[0], maps[1]);
}

inline cudaError_t launch_update7_tma_any(const SimDev &d, const CUtensorMap *maps, int, bool pdl, cudaStream_t s)
{
    return d.noise_on ? launch_update7_tma<true>(d, maps, pdl, s) : launch_update7_tma<false>(d, maps, pdl, s);
}

} // namespace lbm
