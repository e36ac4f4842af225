// Shared definitions of the CUDA library: D2Q9 lattice constants, the Philox
// generator, the device-resident scalar block and the launch descriptor.
//
// Lattice: D2Q9 (the paper's Sec. II lattice is D2Q7; this library implements
// the D2Q9 analogue). Directions 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1)
// 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1); opposite pairs 1-3, 2-4, 5-7, 6-8.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int NQ = 9;
__host__ __device__ constexpr int ex(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int ey(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5); }
// Weights 4/9, 1/9, 1/36 (D2Q9, c_s^2 = 1/3).
template <typename R>
__host__ __device__ constexpr R wq(int i) { return i == 0 ? R(4) / R(9) : (i <= 4 ? R(1) / R(9) : R(1) / R(36)); }
// Division pairs (Sec. II, "two opposite lattice vectors"): pair p loads
// directions pair_a(p) and pair_b(p) = opp(pair_a(p)).
__host__ __device__ constexpr int pair_a(int p) { return p == 0 ? 1 : (p == 1 ? 2 : (p == 2 ? 5 : 6)); }
__host__ __device__ constexpr int pair_b(int p) { return opp(pair_a(p)); }

static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opp axis");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opp diag");

enum GrowthMode { GROW_NONE = 0, GROW_BULK = 1, GROW_DENSITY = 2, GROW_EDGE = 3, GROW_BAND = 4 };
enum { STREAM_PROLIF = 1u, STREAM_INIT = 2u, STREAM_NOISE = 16u };
enum { ST_FRONT_AT_TOP = 1, ST_STARVED = 2, ST_CAPACITY = 4, ST_TIMEOUT = 8 };

// A division site (node (x, y), opposite pair p) packed into 32 bits:
// y << 17 | x << 2 | p (W, H <= 32768 and W H < 2^30 keep every key below
// 0xFFFFFFFF, the empty marker of the merge tables).
__host__ __device__ __forceinline__ uint32_t pack_key(int x, int y, int p)
{
    return ((uint32_t)y << 17) | ((uint32_t)x << 2) | (uint32_t)p;
}
__host__ __device__ __forceinline__ int key_x(uint32_t k) { return (int)((k >> 2) & 0x7FFFu); }
__host__ __device__ __forceinline__ int key_y(uint32_t k) { return (int)(k >> 17); }
__host__ __device__ __forceinline__ int key_pair(uint32_t k) { return (int)(k & 3u); }

// Fixed-point unit of the exact mass sums: 2^-24 per count.
constexpr double kFixScale = 16777216.0;
constexpr double kFixInv = 5.9604644775390625e-08;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of the
// 4x32 S-box, multipliers 0xD2511F53 / 0xCD9E8D57, key bumped by the Weyl
// constants 0x9E3779B9 / 0xBB67AE85 between rounds.
struct u32x4 {
    uint32_t x, y, z, w;
};

// Round keys of one Philox key: k0 + r * 0x9E3779B9, k1 + r * 0xBB67AE85 for
// r = 0..9. Precomputed once per simulation so that inside kernels they are
// constant operands rather than per-call arithmetic.
struct PhiloxKey {
    uint32_t k0[10], k1[10];
};

__host__ __device__ inline PhiloxKey philox_key(uint32_t k0, uint32_t k1)
{
    PhiloxKey k;
    for (int r = 0; r < 10; ++r) {
        k.k0[r] = k0 + (uint32_t)r * 0x9E3779B9u;
        k.k1[r] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    return k;
}

__host__ __device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, const PhiloxKey &k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32 x 32 -> 64-bit product per multiplier
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c.z;
        c = u32x4{(uint32_t)(p1 >> 32) ^ c.y ^ k.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.k1[r],
                  (uint32_t)p0};
    }
    return c;
}

// Uniform on (0, 1): (v + 1/2) 2^-32, exact in double.
__host__ __device__ __forceinline__ double u01(uint32_t v) { return ((double)v + 0.5) * 2.3283064365386963e-10; }

// ---------------------------------------------------------------------------
// Device-resident scalars of one simulation. Written by the kernels only
// (besides initialisation), read back by the host on demand.
struct DevScalars {
    long long step;
    long long mass_fix;       // active mass M, fixed point
    long long quiescent_fix;  // mass behind the rear wall
    unsigned long long mass_accum; // per-step accumulator of the update kernel
    long long S1, S2;
    long long ns_last, ns_total, div_total, starved_steps, cand_last, events_last;
    long long node_updates;
    double carry, hbar, w, clip_mass;
    int y_r, y_copy, y_hi, H_top, hmin;
    int maxmass_accum; // highest row holding mass, accumulated by the update kernel
    int status;
    int n_events;      // event-list entries (draw ranks) of the latest step
    // accumulators of the multi-block observer (reset by its last block)
    long long S1_acc, S2_acc;
    int top_acc, low_acc;
    unsigned int obs_done;
    int pad0;
    // proliferation plan for the next step, made by the observer from the
    // state after the latest step and committed by the selector
    long long plan_req;   // n_s = floor(g M / rho_cell + carry)
    long long plan_ns;    // divisions to draw (0 if nothing can be drawn)
    long long plan_kc;    // candidates evaluated by the parallel pass (multiple of 32)
    unsigned long long plan_nwin; // candidate nodes
    double plan_carry;    // carried fraction after this step's n_s
    double acc_ratio;     // candidates per division seen last time
    int plan_ylo;         // first candidate row
    int plan_nwin_zero;   // n_s > 0 but no candidate row
    // the fused planner (k_plan) selects the divisions of the next step at the
    // end of the current one; their statistics are committed by the following
    // k_plan, after the update that applies them has run
    long long pend_req;   // n_s of the selected step
    long long pend_acc;   // divisions selected (<= n_s)
    long long pend_cand;  // candidates drawn up to the n_s-th accept (or the cap)
    double pend_carry;    // carried fraction after that step's n_s
    int pend_nev;         // list entries of the selection (its draw ranks)
    int pend_starved;     // the selection came up short
    int rec_n;            // division records of the next update
    int pad1;
    unsigned long long bar_ctr; // grid-barrier arrivals of k_plan (grows by the grid size per barrier;
                                // zero when a launch starts)
    unsigned int plan_exit;     // k_plan blocks done with the current launch
    int pad3;
    // k_plan scratch: n_s from the mass before any freezing, computed by one
    // block while the others scan the front
    long long spec_req;
    double spec_carry, spec_kcf;
    // failure-detection test hooks (lbm_debug_waits): the clock-cycle budget
    // of every bounded wait (0: the default of about two seconds), and what a
    // test withholds so that waits run out (WAIT_TEST_* bits)
    long long wait_budget;
    int wait_test;
    int pad2;
    // a batch's estimate of this member's planner work (candidates drawn for
    // the latest selection): copied from pend_cand by the batched injection
    // launch, read by the batched planner launches that follow it
    long long plan_work;
};
enum { WAIT_TEST_COPIES = 1, WAIT_TEST_BARRIER = 2 };
// Default budget of the bounded waits: about two seconds at 2 GHz.
constexpr long long kWaitBudget = 4000000000ll;

// Everything a kernel needs to know about one simulation.
struct SimDev {
    void *f[2];          // population copies, [q][y][x] with row pitch Wp: f[b] points at
                         // (0, 0, 0); a stored row spans x = -kXO .. Wp - kXO - 1, where
                         // x = -1 and x = W are ghost copies of columns W - 1 and 0
    uint32_t *mask;      // occupancy bits, [y][MW], MW = ceil(W / 32)
    int32_t *heights;    // h(x), W entries
    DevScalars *sc;
    // proliferation planner
    unsigned long long *htab; // open-addressing table of the selected (node, pair): packed key
                              // in the high word, draw count in the low word; all ones when unused
    int32_t *hlist;      // per selected division (draw rank): its table slot if it was the
                         // first draw of its (node, pair), else -1
    uint32_t *ev_key;    // divisions of step t at [(t & 1) ns_max, ...) by draw rank: packed (node, pair)
    int32_t *ev_count;   // and how often it was drawn (0 for repeats of an earlier rank)
    int32_t *rows0;      // initial occupied rows per column
    int W, H, Wp, MW;
    long long P;         // plane stride in elements (Wp * H)
    int hcap, ns_max;
    // model constants (all derived on the host once, in double)
    double omega, cmu, rho_c, rho_cell, half_cell, growth_rate, rho0, sigma;
    double rho_init, rho_jitter, wall_min_gap, wall_w_factor;
    uint32_t key0, key1, sim;
    PhiloxKey pk;        // round keys of (key0, key1)
    int growth_mode, edge_depth, band_rows, wall_mode, negfix, y_periodic;
    int noise_on;        // sigma != 0
    int inject_in_update; // the selector only lists the divisions; the update kernel adds them
    int upd_ctas;         // CTAs of the TMA-staged update kernel (tiles dealt round-robin)
    uint32_t upd_magic;   // ceil(2^32 / upd_ctas), upd_ctas >= 2: tile / upd_ctas = umulhi(tile, magic)
    int upd_tyl2;         // log2 of the rows per tile of the TMA-staged update
    int *rec_owner;       // per division (selector order): owning CTA of its tile,
    int *rec_k;           // the tile's index among that CTA's tiles,
    int *rec_off;         // and the two pre-stream slots' offsets in the staged box
                          // (the amount is ev_count * rho_cell / 2)
    int *bucket_cnt;      // divisions per CTA of the TMA-staged update (kTmaMaxCtas)
    int *bucket;          // their record indices, kBucketCap per CTA
    // per-block partials of the fused planner (kPlanMaxBlocks each)
    long long *pl_s1, *pl_s2, *pl_mass;
    int *pl_top, *pl_low, *pl_cnt;
    int plan_grid;        // blocks of the fused planner (all co-resident)
    // the same constants rounded to float once on the host, so that no kernel
    // evaluates double arithmetic per node (the FP64 pipe is narrow)
    float f_rho_c, f_omega, f_cmu, f_om1, f_ow0, f_ow1, f_ow5, f_two_sigma;
    // 16-bit storage: the rest-state populations c_k = w_k rho_init, rounded
    // to the 16-bit type (k: 0 rest, 1 axis, 2 diagonal); unused otherwise
    float pop_shift[3];
    int update_grid;     // persistent grid of the update kernel
};

// What the batched TMA-staged update needs to know about one member besides
// its step and window: 128 bytes, built once per batch, copied into shared
// memory together with each tile of that member.
struct __align__(16) MemberConst {
    void *f[2];
    uint32_t *mask;
    DevScalars *sc;
    long long P;
    int W, H, Wp, MW;
    uint32_t key0, key1, sim;
    int negfix;
    float rho_c, om1, ow1, ow5, cmu, two_sigma;
    float pop_shift[3];
    int pad[3];
};
static_assert(sizeof(MemberConst) == 128, "one 128-byte block per member");

// Launchers of one precision (implemented once per storage type).
struct KernelTable {
    int elem_bytes;
    cudaError_t (*fill)(const SimDev &, cudaStream_t);
    cudaError_t (*ghosts)(const SimDev &, cudaStream_t);
    cudaError_t (*scan)(const SimDev &, int cur, cudaStream_t);
    // Per-step kernels read the step t from the device scalars (step t reads
    // population copy t & 1), so a captured step can be replayed unchanged.
    // fused planner: observe the state after the latest update (init: the
    // current state) and select the divisions of the next step
    cudaError_t (*plan)(const SimDev &, int init, cudaStream_t);
    // the selected divisions of the coming step (update kernels without staging)
    cudaError_t (*inject)(const SimDev &, cudaStream_t);
    cudaError_t (*update)(const SimDev &, cudaStream_t);
    cudaError_t (*fields)(const SimDev &, int cur, double *rho, double *ux, double *uy, cudaStream_t);
    int (*plan_blocks_per_sm)(int batch); // of the own planner (0) or the batched one (1)
    int (*update_blocks_per_sm)();
    int update_tile_x; // columns per block of the update kernel
    // TMA-staged update (lbm_update_tma.cuh, for D2Q7 lbm_update7_tma.cuh;
    // null for FP64 storage). maps[b] loads from copy b (box (kTmaBoxX + 8) x
    // (rows per tile + 2) x Q, in stored-row coordinates); maps[2 + b] stores
    // into copy b for the variants that store in bulk (box kTmaBoxX x rows
    // per tile x Q, columns cut at x = W - 1). tma_prepare sets
    // the kernel attributes a launch needs (the first launch does it too);
    // pdl: launch as a programmatic dependent of the preceding kernel.
    cudaError_t (*tma_prepare)(const SimDev &, int variant);
    cudaError_t (*tma_update)(const SimDev &, const CUtensorMap *maps, int variant, bool pdl, cudaStream_t);
    // a staged variant's geometry: rows of one bulk copy's box, rows per
    // tile, CTAs per SM; 0 for a variant the table has, 1 for one that also
    // stores in bulk, -1 for none
    int (*tma_info)(int variant, int *box_rows, int *iter_rows, int *ctas_per_sm);
    // One step's kernels for every simulation of a batch in one launch each:
    // ds, the simulations' SimDev in device memory; bm, nb entries (simulation,
    // block, blocks) of the update's (a multiple of each simulation's column
    // tiles), the injection's or the planner's block table (the planner: one
    // block per simulation, or its own grid, then cooperatively).
    cudaError_t (*batch_inject)(const SimDev *ds, int nslots, int grid, cudaStream_t);
    cudaError_t (*batch_update)(const SimDev *ds, const int4 *bm, int nb, cudaStream_t);
    cudaError_t (*batch_plan)(const SimDev *ds, int nslots, int cap, cudaStream_t);
    // the TMA-staged update of a whole batch (lbm_update_tma_batch.cuh; null
    // where there is none): mc[m] member m's constants, maps[4 m + b] loads its
    // copy b in boxes of (kTmaBoxX + 8) x 4 x 9, maps[4 m + 2 + b] stores into
    // it (tstore) in boxes of kTmaBoxX x 2 x 9; noise: some member has
    // sigma != 0
    cudaError_t (*batch_update_tma)(const SimDev *ds, const MemberConst *mc, const CUtensorMap *maps, int n,
                                    int noise, int tstore, int grid, cudaStream_t);
};

extern const KernelTable kTableF32;
extern const KernelTable kTableF64;
extern const KernelTable kTableF16;
extern const KernelTable kTableBF16;
extern const KernelTable kTableF32Q7; // the triangular D2Q7 lattice
extern const KernelTable kTableF64Q7;

// Records a CUDA error for lbm_last_cuda_error and maps it to an LBM_ERR_* code.
int lbm_record_cuda_error(cudaError_t e);
// Stored columns left of x = 0 (so that tile boxes start at stored column
// 128 k, 16-byte aligned for every storage type): x = -1 is the ghost of
// column W - 1.
constexpr int kXO = 4;
constexpr int kTmaBoxX = 128;
constexpr int kTmaMaxCtas = 2048; // the reciprocal above is exact for tile * upd_ctas < 2^32
constexpr int kBucketCap = 256;    // division records listed per update CTA (more: full scan)
constexpr int kPlanMaxBlocks = 1024;
// The TMA-staged batched update: members one launch takes (its shared-memory
// tables) and CTAs per SM.
constexpr int kTmaBatchMaxSims = 256;
constexpr int kMaxBatchSlots = 1024; // slots of a batch (the staged batched update: kTmaBatchMaxSims)
constexpr int kTmaBatchCtasPerSm = 5;
constexpr int kTmaBatchCtasPerSmStore = 6; // its bulk-store form
constexpr int kTmaBatchChunk = 8;          // consecutive tiles dealt to one CTA of the staged batched update

} // namespace lbm
