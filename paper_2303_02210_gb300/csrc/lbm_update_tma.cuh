// TMA-staged fused update (FP32 storage, walls in y), the fast path of
// App. A steps 1-7 (step 3's divisions are added to the staged tile): the same
// per-node arithmetic as k_update<float>, different data movement.
//
// Each CTA (persistent, CTAS per SM) walks tiles of 128 columns x TY rows of
// the active window, dealt round-robin over the grid. A tile's pre-stream
// populations arrive in shared memory as one 3-D bulk tensor copy of box
// 136 x (TY + 2) x 9: the tile plus 4 stored columns on each side and one row
// above and below, for all nine planes. The stored rows carry ghost copies of
// the periodic neighbours (x = -1 holds column W - 1, x = W holds column 0), so
// the box needs no patching and never starts outside the stored row.
//
// Pipeline: STAGES boxes per CTA. Consumers wait on the stage's `full`
// mbarrier (transaction bytes, suspending rather than spinning), take their
// values into registers and arrive on its `empty` mbarrier; thread 0 refills
// the stage once every warp has arrived. Warps never wait for each other
// otherwise (a CTA-wide barrier only on the tiles that receive divisions).
//
// Thread layout: two warps per tile row, each lane two adjacent columns
// (2 lane, 2 lane + 1 of its warp's 64): unshifted planes are one 8-byte
// shared load for both nodes, planes shifted in x two 4-byte loads; results
// are 8-byte stores (256 contiguous bytes per warp and plane). Both nodes'
// Philox blocks are drawn together before either node is relaxed.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_tma.cuh"

namespace lbm {

constexpr int TMA_TX = kTmaBoxX;   // 128 columns: two warps of 64
constexpr int TMA_LX = TMA_TX + 8; // staged columns x0 - 4 .. x0 + 131
// Divisions of a CTA kept in shared memory (more are read from global memory
// per tile); tiles flagged per CTA.
constexpr int TMA_EV_CAP = 512;
constexpr int TMA_KFLAG_WORDS = 32;
static_assert(kBucketCap <= TMA_EV_CAP, "a full bucket fits in shared memory");
// a stalled copy is given up after about two seconds at 2 GHz
constexpr long long TMA_WAIT_BUDGET = 4000000000ll;
static_assert(kXO % 4 == 0, "tile boxes start on 16-byte boundaries");

template <int TY>
struct TmaGeom {
    static constexpr int NT = 64 * TY;                          // threads: two warps per row
    static constexpr int WARPS = NT / 32;
    static constexpr int LY = TY + 2;
    static constexpr int PLANE = LY * TMA_LX;                   // floats per staged plane
    static constexpr int IN_FLOATS = 9 * PLANE;                 // one box
    static constexpr int STRIDE = (IN_FLOATS + 31) / 32 * 32;   // stage pitch, 128-byte multiple
    static constexpr uint32_t BYTES = (uint32_t)IN_FLOATS * 4u; // bytes one box copy delivers
};

template <int TY, int STAGES>
constexpr size_t tma_smem_bytes()
{
    return 128 + (size_t)STAGES * TmaGeom<TY>::STRIDE * 4 + 16 * STAGES + (size_t)TMA_EV_CAP * 16 +
           TMA_KFLAG_WORDS * 4;
}
static_assert(3 * (tma_smem_bytes<4, 2>() + 1024) <= 228 * 1024, "three CTAs per SM by shared memory");
static_assert(2 * (tma_smem_bytes<4, 3>() + 1024) <= 228 * 1024, "two CTAs per SM by shared memory");

__device__ __forceinline__ float2 lds2(const float *p) { return *reinterpret_cast<const float2 *>(p); }

// The populations two adjacent nodes pull: `b` points at the first node's
// staged plane-0 value (8-byte aligned). Across the rear (REAR) or top (TOP)
// wall a node takes its own opposite population (half-way bounce-back).
template <int PLANE, bool REAR, bool TOP>
__device__ __forceinline__ void pull2(const float *b, float ga[NQ], float gb[NQ])
{
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        const bool own = (ey(i) == 1 && REAR) || (ey(i) == -1 && TOP);
        if (own) {
            const float2 v = lds2(b + opp(i) * PLANE);
            ga[i] = v.x;
            gb[i] = v.y;
        } else if (ex(i) == 0) {
            const float2 v = lds2(b + i * PLANE - ey(i) * TMA_LX);
            ga[i] = v.x;
            gb[i] = v.y;
        } else {
            const float *p = b + i * PLANE - ey(i) * TMA_LX - ex(i);
            ga[i] = p[0];
            gb[i] = p[1];
        }
    }
}

// One node: relaxation (or reversal below rho_c), the negative fix; returns
// the mass the fix added.
template <bool NOISE>
__device__ __forceinline__ float update_node(const float g[NQ], float rho, bool occ, float fo[NQ], const u32x4 &w,
                                             const Consts<float> &cf, int negfix)
{
    if (occ) {
        relax_words<float, NOISE>(g, rho, fo, w, cf);
        return fix_negative<float>(fo, negfix);
    }
    // rho < rho_c: reverse the directions (two-step bounce-back)
#pragma unroll
    for (int i = 0; i < NQ; ++i) fo[i] = g[opp(i)];
    return 0.0f;
}

// CTAS CTAs per SM (registers are capped so that they fit); NOISE: sigma != 0.
template <int TY, int STAGES, int CTAS, bool NOISE>
__global__ void __launch_bounds__(TmaGeom<TY>::NT, CTAS)
    k_update_tma(SimDev d, const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1)
{
    using G = TmaGeom<TY>;
    constexpr int NT = G::NT, PLANE = G::PLANE;
    extern __shared__ __align__(128) float smem_f[];
    // stages on a 128-byte boundary (offset from the array itself, so that
    // every access stays a shared-memory access)
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

    // prologue, which may overlap the end of the planner (programmatic
    // dependent launch): barriers, tensor map, tile flags
    if (tid == 0) {
        s_abort = 0;
        s_nev = 0;
        prefetch_tensormap(&tm0);
        prefetch_tensormap(&tm1);
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], G::WARPS);
        }
        fence_mbar_init();
    }
    if (tid < TMA_KFLAG_WORDS) kflag[tid] = 0u;
    __syncthreads();
    // everything below reads what the planner wrote
    grid_dependency_wait();
    // step t (read from the device, so a captured step replays as is) pulls
    // from copy t & 1 (tensor map tm0 or tm1) and writes the other
    const uint32_t t = (uint32_t)d.sc->step;
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
            for (int i = 0; i < NQ; ++i) fout[i * P + o] = fin[i * P + o];
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
    if (tid == 0)
        while (issued < STAGES && issued < count) issue();

    // App. A step 3 for this CTA: the planner wrote one record per division
    // (the tile's local index among its owner's tiles, the offsets of the two
    // pre-stream slots in the staged box, the amount) and listed the records
    // of each owner CTA in its bucket; read ours (all records if the bucket
    // overflowed).
    const int nev_all = d.inject_in_update ? d.sc->rec_n : 0;
    const int mine = nev_all > 0 ? d.bucket_cnt[blockIdx.x] : 0;
    if (mine <= kBucketCap) {
        for (int j = tid; j < mine; j += NT) {
            const int e = d.bucket[blockIdx.x * kBucketCap + j];
            const int k = d.rec_k[e];
            ev_k[j] = k;
            ev_off[2 * j] = d.rec_off[2 * e];
            ev_off[2 * j + 1] = d.rec_off[2 * e + 1];
            ev_add[j] = d.rec_add[e];
            if (k < 32 * TMA_KFLAG_WORDS) atomicOr(&kflag[k >> 5], 1u << (k & 31));
        }
        if (tid == 0) s_nev = mine;
    } else {
        constexpr int EV_BATCH = 8; // owner words a thread loads before it looks at any
        for (int eb = 0; eb < nev_all; eb += NT * EV_BATCH) {
            int own[EV_BATCH];
#pragma unroll
            for (int j = 0; j < EV_BATCH; ++j) {
                const int e = eb + j * NT + tid;
                own[j] = e < nev_all ? d.rec_owner[e] : -1;
            }
#pragma unroll
            for (int j = 0; j < EV_BATCH; ++j) {
                const int e = eb + j * NT + tid;
                if (own[j] == (int)blockIdx.x) {
                    const int at = atomicAdd(&s_nev, 1);
                    const int k = d.rec_k[e];
                    if (at < TMA_EV_CAP) {
                        ev_k[at] = k;
                        ev_off[2 * at] = d.rec_off[2 * e];
                        ev_off[2 * at + 1] = d.rec_off[2 * e + 1];
                        ev_add[at] = d.rec_add[e];
                    }
                    if (k < 32 * TMA_KFLAG_WORDS) atomicOr(&kflag[k >> 5], 1u << (k & 31));
                }
            }
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
        if (!dead && !mbar_wait_bounded(&full[s], parity, TMA_WAIT_BUDGET)) {
            dead = true;
            atomicOr(&s_abort, 1);
        }
        // divisions of this tile, added to the staged pre-stream slots
        const bool has_ev =
            nev > 0 && (ev_overflow || k >= 32 * TMA_KFLAG_WORDS || ((kflag[k >> 5] >> (k & 31)) & 1u));
        if (has_ev) { // uniform across the CTA
            if (!ev_overflow) {
                for (int i = tid; i < nev; i += NT)
                    if (ev_k[i] == k) {
                        stage[ev_off[2 * i]] += ev_add[i];
                        stage[ev_off[2 * i + 1]] += ev_add[i];
                    }
            } else {
                for (int e = tid; e < nev_all; e += NT)
                    if (d.rec_owner[e] == (int)blockIdx.x && d.rec_k[e] == k) {
                        stage[d.rec_off[2 * e]] += d.rec_add[e];
                        stage[d.rec_off[2 * e + 1]] += d.rec_add[e];
                    }
            }
            fence_proxy_async_smem(); // before a later bulk copy overwrites them
            __syncthreads();
        }
        // the pulled populations of this thread's two nodes (rows past the
        // active window hold no mass and are skipped; warp-uniform)
        const int y = y0 + row;
        const bool active = y < y_hi;
        float ga[NQ], gb[NQ];
        if (active) {
            const float *b = stage + (row + 1) * TMA_LX + cl + 4;
            const bool rear = y - 1 < y_r, top = y + 1 >= H; // half-way bounce-back walls
            if (!rear && !top)
                pull2<PLANE, false, false>(b, ga, gb);
            else if (!top)
                pull2<PLANE, true, false>(b, ga, gb);
            else if (!rear)
                pull2<PLANE, false, true>(b, ga, gb);
            else
                pull2<PLANE, true, true>(b, ga, gb);
        }
        // the stage may be refilled (by the async proxy) once every warp has
        // arrived: order this thread's shared-memory reads before that
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (tid == 0 && issued < count) {
            // refill this stage once every warp has its values
            if (!dead && !mbar_wait_bounded(&empty[s], parity, TMA_WAIT_BUDGET)) {
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
            for (int i = 1; i < NQ; ++i) {
                rhoa = rhoa + ga[i];
                rhob = rhob + gb[i];
            }
            const bool occa = oka && rhoa >= rho_c, occb = okb && rhob >= rho_c;
            if (__all_sync(0xffffffffu, occa && occb)) {
                // the bulk: all 64 nodes of the warp's segment are occupied
                const uint32_t n = (uint32_t)(y * W + x);
                float fa[NQ], fb[NQ];
                relax_words<float, NOISE>(ga, rhoa, fa, NOISE ? noise_block(n, t, d) : u32x4{0u, 0u, 0u, 0u}, cf);
                relax_words<float, NOISE>(gb, rhob, fb, NOISE ? noise_block(n + 1u, t, d) : u32x4{0u, 0u, 0u, 0u},
                                          cf);
                float mn = fminf(fa[0], fb[0]);
#pragma unroll
                for (int i = 1; i < NQ; ++i) mn = fminf(mn, fminf(fa[i], fb[i]));
                float adda = 0.0f, addb = 0.0f;
                if (__any_sync(0xffffffffu, mn < 0.0f)) {
                    adda = fix_negative<float>(fa, negfix);
                    addb = fix_negative<float>(fb, negfix);
                    clip += adda + addb;
                }
                if ((lane & 15) == 0) d.mask[(long long)y * d.MW + (x0 >> 5) + 2 * half + (lane >> 4)] = 0xffffffffu;
                float *o = fout + (long long)y * Wp + x;
#pragma unroll
                for (int i = 0; i < NQ; ++i) *reinterpret_cast<float2 *>(o + i * P) = make_float2(fa[i], fb[i]);
                const int xw = x0 + 64 * half; // first column of the warp
                if (xw == 0 || xw + 63 == W - 1) { // a warp at the lattice edge: ghost copies
                    if (x == 0) {
#pragma unroll
                        for (int i = 0; i < NQ; ++i) o[i * P + W] = fa[i];
                    }
                    if (x + 1 == W - 1) {
#pragma unroll
                        for (int i = 0; i < NQ; ++i) o[i * P + 1 - W] = fb[i];
                    }
                }
                const float roa = rhoa + adda, rob = rhob + addb;
                mass += fix24<float>(roa) + fix24<float>(rob);
                if (roa != 0.0f || rob != 0.0f) maxrow = y;
            } else {
                u32x4 wa{0u, 0u, 0u, 0u}, wb{0u, 0u, 0u, 0u};
                if (NOISE && (occa || occb)) {
                    const uint32_t n = (uint32_t)(y * W + x);
                    wa = noise_block(n, t, d);
                    wb = noise_block(n + 1u, t, d);
                }
                float fa[NQ], fb[NQ];
                const float adda = update_node<NOISE>(ga, rhoa, occa, fa, wa, cf, negfix);
                const float addb = update_node<NOISE>(gb, rhob, occb, fb, wb, cf, negfix);
                // occupancy bits: lanes 0-15 hold one 32-column word, lanes 16-31 the next
                unsigned v = ((unsigned)occa | ((unsigned)occb << 1)) << (2 * (lane & 15));
                v |= __shfl_xor_sync(0xffffffffu, v, 1);
                v |= __shfl_xor_sync(0xffffffffu, v, 2);
                v |= __shfl_xor_sync(0xffffffffu, v, 4);
                v |= __shfl_xor_sync(0xffffffffu, v, 8);
                const int word = (x0 >> 5) + 2 * half + (lane >> 4);
                if ((lane & 15) == 0 && word < d.MW) d.mask[(long long)y * d.MW + word] = v;
                float *o = fout + (long long)y * Wp + x;
                if (okb) {
    #pragma unroll
                    for (int i = 0; i < NQ; ++i) *reinterpret_cast<float2 *>(o + i * P) = make_float2(fa[i], fb[i]);
                } else if (oka) { // odd W: the last column alone (x = W is the ghost)
    #pragma unroll
                    for (int i = 0; i < NQ; ++i) o[i * P] = fa[i];
                }
                // ghost copies of the edge columns for the next step's boxes
                if (x == 0) {
    #pragma unroll
                    for (int i = 0; i < NQ; ++i) o[i * P + W] = fa[i];
                }
                if (x == W - 1) {
    #pragma unroll
                    for (int i = 0; i < NQ; ++i) o[i * P - W] = fa[i];
                }
                if (x + 1 == W - 1) {
    #pragma unroll
                    for (int i = 0; i < NQ; ++i) o[i * P + 1 - W] = fb[i];
                }
                // populations are non-negative after every step, so a node holds
                // mass iff their sum (rho + what the fix added) is non-zero
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
            mbar_wait_bounded(&full[k % STAGES], (uint32_t)((k / STAGES) & 1), TMA_WAIT_BUDGET);
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
template <int TY, int STAGES, int CTAS, bool NOISE>
cudaError_t prepare_update_tma_variant()
{
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !attr[dev]) {
        e = cudaFuncSetAttribute(k_update_tma<TY, STAGES, CTAS, NOISE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tma_smem_bytes<TY, STAGES>());
        if (e != cudaSuccess) return e;
        if (dev < 64) attr[dev] = true;
    }
    return cudaSuccess;
}

inline cudaError_t prepare_update_tma(const SimDev &d, int variant)
{
    if (variant == 1)
        return d.noise_on ? prepare_update_tma_variant<4, 3, 2, true>() : prepare_update_tma_variant<4, 3, 2, false>();
    return d.noise_on ? prepare_update_tma_variant<4, 2, 3, true>() : prepare_update_tma_variant<4, 2, 3, false>();
}

template <int TY, int STAGES, int CTAS, bool NOISE>
cudaError_t launch_update_tma_variant(const SimDev &d, const CUtensorMap *maps, bool pdl, cudaStream_t s)
{
    cudaError_t e = prepare_update_tma_variant<TY, STAGES, CTAS, NOISE>();
    if (e != cudaSuccess) return e;
    // maps[b] loads from population copy b. Launched as a programmatic
    // dependent of the planner: its CTAs may start (and run the prologue)
    // before the planner has finished, and wait for it in grid_dependency_wait.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)d.upd_ctas); // at most CTAS per SM
    cfg.blockDim = dim3(TmaGeom<TY>::NT);
    cfg.dynamicSmemBytes = tma_smem_bytes<TY, STAGES>();
    cfg.stream = s;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    la[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = la;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_update_tma<TY, STAGES, CTAS, NOISE>, d, maps[0], maps[1]);
}

// variant 0: two staged tiles per CTA, three CTAs per SM; variant 1: three
// staged tiles per CTA, two CTAs per SM. Both use tiles of 4 rows.
constexpr int tma_rows(int /*variant*/) { return 4; }
constexpr int tma_ctas_per_sm(int variant) { return variant == 1 ? 2 : 3; }

inline cudaError_t launch_update_tma(const SimDev &d, const CUtensorMap *maps, int variant, bool pdl, cudaStream_t s)
{
    if (variant == 1)
        return d.noise_on ? launch_update_tma_variant<4, 3, 2, true>(d, maps, pdl, s)
                          : launch_update_tma_variant<4, 3, 2, false>(d, maps, pdl, s);
    return d.noise_on ? launch_update_tma_variant<4, 2, 3, true>(d, maps, pdl, s)
                      : launch_update_tma_variant<4, 2, 3, false>(d, maps, pdl, s);
}

} // namespace lbm
