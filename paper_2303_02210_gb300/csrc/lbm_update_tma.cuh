// TMA-staged fused update (FP32 or 16-bit storage, walls in y), the fast path
// of App. A steps 1-7 (step 3's divisions are added to the staged tile): the
// same per-node arithmetic as k_update, different data movement.
//
// Each CTA (persistent, CTAS per SM) walks tiles of 128 columns x TY rows of
// the active window, dealt round-robin over the grid. A tile's pre-stream
// populations arrive in shared memory as one 3-D bulk tensor copy of box
// 136 x (TY + 2) x 9 elements: the tile plus 4 stored columns on each side and one row
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
// (2 lane, 2 lane + 1 of its warp's 64): unshifted planes are one paired
// shared load for both nodes, planes shifted in x two scalar loads; results
// are paired stores (64 contiguous elements per warp and plane). Both nodes'
// Philox blocks are drawn together before either node is relaxed.
//
// 16-bit storage (FP16, BF16; the deviation from the rest state, see Pop):
// the staged values are decoded to FP32 as they are read, the results are
// encoded two at a time (one packed conversion per plane and node pair), and
// a division is added to a staged slot as decode, FP32 add, encode, which
// rounds exactly as k_inject does in global memory. The boxes are half as
// large, so twice as many are kept in flight per CTA.
#pragma once

#include <type_traits>

#include "lbm_kernels.cuh"
#include "lbm_pair.cuh"
#include "lbm_tma.cuh"

namespace lbm {

constexpr int TMA_TX = kTmaBoxX;   // 128 columns: two warps of 64
constexpr int TMA_LX = TMA_TX + 8; // staged columns x0 - 4 .. x0 + 131
// Divisions of a CTA kept in shared memory (more are read from global memory
// per tile); tiles flagged per CTA.
constexpr int TMA_EV_CAP = 128;
constexpr int TMA_KFLAG_WORDS = 32;
static_assert(kXO % 4 == 0, "tile boxes start on 16-byte boundaries");

template <typename S, int TY>
struct TmaGeom {
    static constexpr int NT = 64 * TY;                                 // threads: two warps per row
    static constexpr int WARPS = NT / 32;
    static constexpr int LY = TY + 2;
    static constexpr int PLANE = LY * TMA_LX;                          // elements per staged plane
    static constexpr int IN_ELEMS = 9 * PLANE;                         // one box
    static constexpr int STRIDE = (IN_ELEMS * (int)sizeof(S) + 127) / 128 * 128 / (int)sizeof(S); // stage pitch
    static constexpr uint32_t BYTES = (uint32_t)IN_ELEMS * (uint32_t)sizeof(S); // one box copy delivers
};

// (TSTORE: an output tile [plane][TY][128] more, for bulk tensor stores)
template <typename S, int TY, int STAGES, bool TSTORE = false>
constexpr size_t tma_smem_bytes()
{
    return 128 + (size_t)STAGES * TmaGeom<S, TY>::STRIDE * sizeof(S) + (TSTORE ? (size_t)9 * TY * TMA_TX * sizeof(S) : 0) +
           16 * STAGES + (size_t)TMA_EV_CAP * 16 + TMA_KFLAG_WORDS * 4;
}

// Configurations. Variant 0: tiles of two rows, 128 threads, five CTAs per
// SM with two stages each (FP32: 20 warps, ten tiles in flight per SM), six
// CTAs with two stages for 16-bit storage (its boxes are half the bytes;
// measured at 8192 x 2048 FP16: 0.452 of the copy peak against 0.436 with
// five CTAs of four stages; seven CTAs 0.246); variant 1: tiles of four
// rows, 256 threads, three CTAs per SM (24 warps, six tiles). Variant 0 gave
// 81.0 against 85.1 us per step on the 4096 x 2048 FP32 workload (the
// two-row boxes re-read more halo rows from the L2, but more, shorter tiles
// keep more copies in flight). Variant 2 (FP32 only): variant 0's tiles, the
// results gathered in a shared output tile and written by one bulk tensor
// store per tile instead of per-lane stores; one stage per CTA and six CTAs
// per SM (the kernel is latency-bound: more warps beat a second stage; per
// step at 4096 x 2048: 71.7 us against 73.2 with four CTAs of two stages,
// 74.7 with five of one, 72.4 with seven of one). (A 16-bit tile starts 4
// elements = 8 bytes into a 16-byte unit, and a bulk tensor store must start
// on a 16-byte boundary.)
template <typename S>
struct TmaCfg {
    static constexpr int TY0 = 2, CTAS0 = sizeof(S) == 4 ? 5 : 6, STAGES0 = sizeof(S) == 4 ? 2 : 2;
    static constexpr int TY1 = 4, CTAS1 = 3, STAGES1 = sizeof(S) == 4 ? 2 : 4;
    static constexpr int TY2 = 2, CTAS2 = 6, STAGES2 = 1;
};
static_assert(6 * (tma_smem_bytes<float, 2, 1, true>() + 1024) <= 228 * 1024, "six CTAs per SM by shared memory");
static_assert(5 * (tma_smem_bytes<float, 2, 2>() + 1024) <= 228 * 1024, "five CTAs per SM by shared memory");
static_assert(3 * (tma_smem_bytes<float, 4, 2>() + 1024) <= 228 * 1024, "three CTAs per SM by shared memory");
static_assert(6 * (tma_smem_bytes<__half, 2, 2>() + 1024) <= 228 * 1024, "six CTAs per SM by shared memory");
static_assert(3 * (tma_smem_bytes<__half, 4, 4>() + 1024) <= 228 * 1024, "three CTAs per SM by shared memory");

// Two adjacent stored elements as one access.
template <typename S> struct Pair2;
template <> struct Pair2<float> { using T = float2; };
template <> struct Pair2<__half> { using T = __half2; };
template <> struct Pair2<__nv_bfloat16> { using T = __nv_bfloat162; };

// Decodes the pair at `p` (aligned to the pair) of plane class q.
template <typename S>
__device__ __forceinline__ void ld_pair(const S *p, int q, const Pop<S> &pc, float &a, float &b)
{
    const typename Pair2<S>::T v = *reinterpret_cast<const typename Pair2<S>::T *>(p);
    a = pc.ld(v.x, q);
    b = pc.ld(v.y, q);
}

// Encodes (a, b) of plane q as one pair (one packed conversion for 16 bits;
// each element rounds as Pop::st would).
template <typename S>
__device__ __forceinline__ typename Pair2<S>::T enc_pair(float a, float b, int q, const Pop<S> &pc)
{
    if constexpr (sizeof(S) == 4) {
        return make_float2(a, b);
    } else if constexpr (std::is_same<S, __half>::value) {
        return __floats2half2_rn(a - pc.shift(q), b - pc.shift(q));
    } else {
        return __floats2bfloat162_rn(a - pc.shift(q), b - pc.shift(q));
    }
}

// Decodes a stored pair of plane class q to FP32 (FP16: one packed conversion
// and one packed add of the shift; per element exactly Pop::ld).
template <typename S>
__device__ __forceinline__ float2 dec_pair(typename Pair2<S>::T v, int q, const Pop<S> &pc)
{
    if constexpr (sizeof(S) == 4) {
        return v;
    } else if constexpr (std::is_same<S, __half>::value) {
        return add2(__half22float2(v), f2(pc.shift(q)));
    } else {
        return make_float2(pc.ld(v.x, q), pc.ld(v.y, q)); // (one mixed-precision add each)
    }
}

// Encodes a pair of plane q (per element exactly Pop::st).
template <typename S>
__device__ __forceinline__ typename Pair2<S>::T enc_pair2(float2 f, int q, const Pop<S> &pc)
{
    if constexpr (sizeof(S) == 4) {
        return f;
    } else if constexpr (std::is_same<S, __half>::value) {
        return __float22half2_rn(sub2(f, f2(pc.shift(q))));
    } else {
        return __float22bfloat162_rn(sub2(f, f2(pc.shift(q))));
    }
}

// pull2 for a pair held as float2 per direction (the .x node and the .y node).
template <typename S, int PLANE, bool REAR, bool TOP>
__device__ __forceinline__ void pull2p(const S *b, float2 g[NQ], const Pop<S> &pc)
{
    using P2 = typename Pair2<S>::T;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        const bool own = (ey(i) == 1 && REAR) || (ey(i) == -1 && TOP);
        P2 v;
        if (own) {
            v = *reinterpret_cast<const P2 *>(b + opp(i) * PLANE);
        } else if (ex(i) == 0) {
            v = *reinterpret_cast<const P2 *>(b + i * PLANE - ey(i) * TMA_LX);
        } else {
            const S *p = b + i * PLANE - ey(i) * TMA_LX - ex(i);
            v.x = p[0];
            v.y = p[1];
        }
        g[i] = dec_pair<S>(v, i, pc);
    }
}

// Stores a node pair from float2 populations; with 16-bit storage m is the
// pair's mass as stored (the decoded stored values summed in index order).
template <typename S>
__device__ __forceinline__ void store_pair(S *o, long long P, const float2 f[NQ], const Pop<S> &pc, float2 &m)
{
    using P2 = typename Pair2<S>::T;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        const P2 v = enc_pair2<S>(f[i], i, pc);
        *reinterpret_cast<P2 *>(o + i * P) = v;
        if constexpr (Pop<S>::kShifted) {
            const float2 dv = dec_pair<S>(v, i, pc);
            m = i == 0 ? dv : add2(m, dv);
        }
    }
}

// The populations two adjacent nodes pull: `b` points at the first node's
// staged plane-0 value (aligned to a pair). Across the rear (REAR) or top
// (TOP) wall a node takes its own opposite population (half-way bounce-back).
template <typename S, int PLANE, bool REAR, bool TOP>
__device__ __forceinline__ void pull2(const S *b, float ga[NQ], float gb[NQ], const Pop<S> &pc)
{
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        const bool own = (ey(i) == 1 && REAR) || (ey(i) == -1 && TOP);
        if (own) {
            ld_pair<S>(b + opp(i) * PLANE, i, pc, ga[i], gb[i]);
        } else if (ex(i) == 0) {
            ld_pair<S>(b + i * PLANE - ey(i) * TMA_LX, i, pc, ga[i], gb[i]);
        } else {
            const S *p = b + i * PLANE - ey(i) * TMA_LX - ex(i);
            ga[i] = pc.ld(p[0], i);
            gb[i] = pc.ld(p[1], i);
        }
    }
}

// Stores the results of a node pair (columns x, x + 1 at `o`), or of the first
// node alone if !both. With 16-bit storage, ma and mb are the nodes' masses as
// stored: the decoded values summed in index order (as in k_update).
template <typename S>
__device__ __forceinline__ void store_nodes(S *o, long long P, const float fa[NQ], const float fb[NQ], bool both,
                                            const Pop<S> &pc, float &ma, float &mb)
{
    ma = mb = 0.0f;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        if (both) {
            const typename Pair2<S>::T v = enc_pair<S>(fa[i], fb[i], i, pc);
            *reinterpret_cast<typename Pair2<S>::T *>(o + i * P) = v;
            if constexpr (Pop<S>::kShifted) {
                const float da = pc.ld(v.x, i), db = pc.ld(v.y, i);
                ma = i == 0 ? da : ma + da;
                mb = i == 0 ? db : mb + db;
            }
        } else {
            const S v = pc.st(fa[i], i);
            o[i * P] = v;
            if constexpr (Pop<S>::kShifted) {
                const float da = pc.ld(v, i);
                ma = i == 0 ? da : ma + da;
            }
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

// CTAS CTAs per SM (registers are capped so that they fit); NOISE: sigma != 0;
// TSTORE: results leave through a shared output tile and one bulk tensor
// store per tile (ts0 / ts1: copy 0 / 1 as [plane][row][stored column] with
// the columns cut at x = W - 1, boxes of 128 x TY x 9), else per-lane stores.
template <typename S, int TY, int STAGES, int CTAS, bool NOISE, bool TSTORE>
__global__ void __launch_bounds__(TmaGeom<S, TY>::NT, CTAS)
    k_update_tma(SimDev d, const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1,
                 const __grid_constant__ CUtensorMap ts0, const __grid_constant__ CUtensorMap ts1)
{
    static_assert(!TSTORE || sizeof(S) == 4, "bulk tensor stores of 16-bit tiles would start off a 16-byte boundary");
    using G = TmaGeom<S, TY>;
    constexpr int NT = G::NT, PLANE = G::PLANE;
    const Pop<S> pc(d);
    extern __shared__ __align__(128) float smem_f[];
    // stages on a 128-byte boundary (offset from the array itself, so that
    // every access stays a shared-memory access)
    S *s_in = reinterpret_cast<S *>(smem_f + ((128u - (smem_u32(smem_f) & 127u)) & 127u) / 4u);
    S *s_out = s_in + STAGES * G::STRIDE; // the output tile (TSTORE), on a 128-byte boundary
    uint64_t *full = reinterpret_cast<uint64_t *>(s_out + (TSTORE ? 9 * TY * TMA_TX : 0));
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
        if (TSTORE) {
            prefetch_tensormap(&ts0);
            prefetch_tensormap(&ts1);
        }
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
    // bounded waits: the budget (a failure-detection test shortens it and may
    // withhold the bulk copies, so that the first wait of every thread runs out)
    const long long budget = d.sc->wait_budget > 0 ? d.sc->wait_budget : kWaitBudget;
    const bool withhold = (d.sc->wait_test & WAIT_TEST_COPIES) != 0;
    const int cur = (int)(t & 1u);
    const CUtensorMap *tm = cur ? &tm1 : &tm0;
    const CUtensorMap *ts = cur ? &ts0 : &ts1; // (the copy this step writes)
    const S *__restrict__ fin = (const S *)d.f[cur];
    S *__restrict__ fout = (S *)d.f[cur ^ 1];
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
    if (tid == 0 && !withhold)
        while (issued < STAGES && issued < count) issue();

    // App. A step 3 for this CTA: the planner wrote one record per division
    // (the tile's local index among its owner's tiles, the offsets of the two
    // pre-stream slots in the staged box; the amount follows from the event
    // count) and listed the records of each owner CTA in its bucket; read
    // ours (all records if the bucket overflowed).
    const int nev_all = d.inject_in_update ? d.sc->rec_n : 0;
    // the amount of division e: count * rho_cell / 2 (the event list of step
    // t; the address is formed at each use, so that nothing more stays live
    // through the tile loop)
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
                        ev_add[at] = amount(e);
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
        S *stage = s_in + s * G::STRIDE;
        if (!dead && !mbar_wait_bounded(&full[s], parity, budget)) {
            dead = true;
            atomicOr(&s_abort, 1);
        }
        // divisions of this tile, added to the staged pre-stream slots
        const bool has_ev =
            nev > 0 && (ev_overflow || k >= 32 * TMA_KFLAG_WORDS || ((kflag[k >> 5] >> (k & 31)) & 1u));
        if (has_ev) { // uniform across the CTA
            // (slot offset / PLANE is the plane, hence the weight class)
            auto add_slot = [&](int off, float a) {
                stage[off] = pc.st(pc.ld(stage[off], off / PLANE) + a, off / PLANE);
            };
            if (!ev_overflow) {
                for (int i = tid; i < nev; i += NT)
                    if (ev_k[i] == k) {
                        add_slot(ev_off[2 * i], ev_add[i]);
                        add_slot(ev_off[2 * i + 1], ev_add[i]);
                    }
            } else {
                for (int e = tid; e < nev_all; e += NT)
                    if (d.rec_owner[e] == (int)blockIdx.x && d.rec_k[e] == k) {
                        const float a = amount(e);
                        add_slot(d.rec_off[2 * e], a);
                        add_slot(d.rec_off[2 * e + 1], a);
                    }
            }
            fence_proxy_async_smem(); // before a later bulk copy overwrites them
            __syncthreads();
        }
        // the pulled populations of this thread's two nodes (rows past the
        // active window hold no mass and are skipped; warp-uniform)
        const int y = y0 + row;
        const bool active = y < y_hi;
        float2 g2[NQ]; // (first node, second node) per direction
        if (active) {
            const S *b = stage + (row + 1) * TMA_LX + cl + 4;
            const bool rear = y - 1 < y_r, top = y + 1 >= H; // half-way bounce-back walls
            if (!rear && !top)
                pull2p<S, PLANE, false, false>(b, g2, pc);
            else if (!top)
                pull2p<S, PLANE, true, false>(b, g2, pc);
            else if (!rear)
                pull2p<S, PLANE, false, true>(b, g2, pc);
            else
                pull2p<S, PLANE, true, true>(b, g2, pc);
        }
        // the stage may be refilled (by the async proxy) once every warp has
        // arrived: order this thread's shared-memory reads before that
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (tid == 0 && issued < count && !withhold) {
            // refill this stage once every warp has its values
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
            // Eq. 1 density of both nodes (index order)
            const float2 rho2 = rho_pair(g2);
            const float rhoa = rho2.x, rhob = rho2.y;
            const bool occa = oka && rhoa >= rho_c, occb = okb && rhob >= rho_c;
            if (__all_sync(0xffffffffu, occa && occb)) {
                // the bulk: all 64 nodes of the warp's segment are occupied;
                // both nodes at once in packed FP32 (lbm_pair.cuh)
                const uint32_t n = (uint32_t)(y * W + x);
                const u32x4 wa = NOISE ? noise_block(n, t, d) : u32x4{0u, 0u, 0u, 0u};
                const u32x4 wb = NOISE ? noise_block(n + 1u, t, d) : u32x4{0u, 0u, 0u, 0u};
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
                if ((lane & 15) == 0) d.mask[(long long)y * d.MW + (x0 >> 5) + 2 * half + (lane >> 4)] = 0xffffffffu;
                S *o = fout + (long long)y * Wp + x;
                float2 m2 = f2(0.0f);
                if constexpr (TSTORE) {
#pragma unroll
                    for (int i = 0; i < NQ; ++i) res[i] = f2o[i];
                } else {
                    store_pair<S>(o, P, f2o, pc, m2);
                }
                const int xw = x0 + 64 * half; // first column of the warp
                if (xw == 0 || xw + 63 == W - 1) { // a warp at the lattice edge: ghost copies
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
                S *o = fout + (long long)y * Wp + x;
                float ma = 0.0f, mb = 0.0f;
                // (odd W: the last column alone, x = W is the ghost)
                if constexpr (TSTORE) {
#pragma unroll
                    for (int i = 0; i < NQ; ++i) res[i] = make_float2(fa[i], fb[i]);
                } else {
                    if (oka) store_nodes<S>(o, P, fa, fb, okb, pc, ma, mb);
                }
                // ghost copies of the edge columns for the next step's boxes
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
                // populations are non-negative after every step, so a node holds
                // mass iff their sum (rho + what the fix added; with 16-bit
                // storage the stored values' sum) is non-zero
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
            fence_proxy_async_smem(); // the async proxy reads what these threads wrote
            __syncthreads();
            if (tid == 0) {
                tma_store_3d(ts, x0 + kXO, y0, 0, s_out);
                bulk_commit();
            }
        }
        tx += dtx;
        ty += dty;
        if (tx >= ncx) {
            tx -= ncx;
            ++ty;
        }
    }
    if (TSTORE && tid == 0) bulk_wait_all(); // the last tiles' stores are done before the CTA exits
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
template <typename S, int TY, int STAGES, int CTAS, bool NOISE, bool TSTORE>
cudaError_t prepare_update_tma_variant()
{
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !attr[dev]) {
        e = cudaFuncSetAttribute(k_update_tma<S, TY, STAGES, CTAS, NOISE, TSTORE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tma_smem_bytes<S, TY, STAGES, TSTORE>());
        if (e != cudaSuccess) return e;
        if (dev < 64) attr[dev] = true;
    }
    return cudaSuccess;
}

// maps[b] loads from population copy b, maps[2 + b] stores into it (TSTORE).
// Launched as a programmatic dependent of the planner: its CTAs may start
// (and run the prologue) before the planner has finished, and wait for it in
// grid_dependency_wait.
template <typename S, int TY, int STAGES, int CTAS, bool NOISE, bool TSTORE>
cudaError_t launch_update_tma_variant(const SimDev &d, const CUtensorMap *maps, bool pdl, cudaStream_t s)
{
    cudaError_t e = prepare_update_tma_variant<S, TY, STAGES, CTAS, NOISE, TSTORE>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)d.upd_ctas); // at most CTAS per SM
    cfg.blockDim = dim3(TmaGeom<S, TY>::NT);
    cfg.dynamicSmemBytes = tma_smem_bytes<S, TY, STAGES, TSTORE>();
    cfg.stream = s;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    la[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = la;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_update_tma<S, TY, STAGES, CTAS, NOISE, TSTORE>, d, maps[0], maps[1],
                              maps[TSTORE ? 2 : 0], maps[TSTORE ? 3 : 1]);
}

template <typename S, bool NOISE>
cudaError_t prepare_update_tma_noise(int variant)
{
    using C = TmaCfg<S>;
    if (variant == 1) return prepare_update_tma_variant<S, C::TY1, C::STAGES1, C::CTAS1, NOISE, false>();
    if constexpr (sizeof(S) == 4)
        if (variant == 2) return prepare_update_tma_variant<S, C::TY2, C::STAGES2, C::CTAS2, NOISE, true>();
    return prepare_update_tma_variant<S, C::TY0, C::STAGES0, C::CTAS0, NOISE, false>();
}

template <typename S>
cudaError_t prepare_update_tma(const SimDev &d, int variant)
{
    return d.noise_on ? prepare_update_tma_noise<S, true>(variant) : prepare_update_tma_noise<S, false>(variant);
}

template <typename S, bool NOISE>
cudaError_t launch_update_tma_noise(const SimDev &d, const CUtensorMap *maps, int variant, bool pdl, cudaStream_t s)
{
    using C = TmaCfg<S>;
    if (variant == 1) return launch_update_tma_variant<S, C::TY1, C::STAGES1, C::CTAS1, NOISE, false>(d, maps, pdl, s);
    if constexpr (sizeof(S) == 4)
        if (variant == 2)
            return launch_update_tma_variant<S, C::TY2, C::STAGES2, C::CTAS2, NOISE, true>(d, maps, pdl, s);
    return launch_update_tma_variant<S, C::TY0, C::STAGES0, C::CTAS0, NOISE, false>(d, maps, pdl, s);
}

template <typename S>
cudaError_t launch_update_tma(const SimDev &d, const CUtensorMap *maps, int variant, bool pdl, cudaStream_t s)
{
    return d.noise_on ? launch_update_tma_noise<S, true>(d, maps, variant, pdl, s)
                      : launch_update_tma_noise<S, false>(d, maps, variant, pdl, s);
}

// Geometry of a variant for the host: rows of one bulk copy's box, rows per
// tile, CTAs per SM; 0 for a variant of this kernel, -1 for none.
// (1: the variant also stores through bulk tensor copies, which want the
// store maps)
template <typename S>
int tile_variant_info(int variant, int *box_rows, int *iter_rows, int *ctas_per_sm)
{
    using C = TmaCfg<S>;
    if (variant == 2 && sizeof(S) == 4) {
        *iter_rows = C::TY2;
        *box_rows = C::TY2 + 2;
        *ctas_per_sm = C::CTAS2;
        return 1;
    }
    if (variant != 0 && variant != 1) return -1;
    *iter_rows = variant == 1 ? C::TY1 : C::TY0;
    *box_rows = *iter_rows + 2;
    *ctas_per_sm = variant == 1 ? C::CTAS1 : C::CTAS0;
    return 0;
}

} // namespace lbm
