// TMA-staged fused update (FP32 storage, walls in y), the fast path of
// App. A steps 1, 2, 4-7: same arithmetic as k_update<float>, different data
// movement.
//
// Each CTA (persistent) walks tiles of TX columns x TY rows of the
// active window. A tile's pre-stream populations arrive in shared memory as one
// 3-D bulk tensor copy of box (TX + 8) x (TY + 2) x 9: the tile plus 4 aligned
// columns on each side and one row above and below, for all nine planes.
// Copies complete on an mbarrier; a CTA issues the copy of its next tile as
// soon as its threads hold the current one in registers, so the copy overlaps
// the compute. Coordinates outside the lattice (x < 0, y < 0, y >= H) arrive as
// zeros; for the two tiles at the ends of a row band the periodic wrap in x is
// patched into the staged tile (the column just outside the lattice on each
// side). Each pulled value is then one shared-memory load at a compile-time
// offset from the node's own position. One warp takes one row of a tile, one
// lane four adjacent columns: aligned planes come in as one 16-byte shared
// load, planes shifted in x as one 16-byte and one 4-byte load; results go
// straight from registers to global memory as 16-byte stores (512 contiguous
// bytes per warp and plane). Two CTAs share an SM.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_tma.cuh"

namespace lbm {

constexpr int TMA_TX = 128;                                      // 32 lanes x 4 columns
constexpr int TMA_TY = 8;                                        // one warp per row
constexpr int TMA_NT = 32 * TMA_TY;
constexpr int TMA_LX = TMA_TX + 8;
constexpr int TMA_LY = TMA_TY + 2;
constexpr int TMA_IN_FLOATS = 9 * TMA_LY * TMA_LX;             // one box
constexpr int TMA_IN_STRIDE = (TMA_IN_FLOATS + 31) / 32 * 32;   // stage pitch, 128-byte multiple
constexpr uint32_t TMA_IN_BYTES = (uint32_t)TMA_IN_FLOATS * 4u; // bytes one box copy delivers
// Slot additions (two per division) a CTA keeps in shared memory for its
// staged tiles (more are read from global memory per tile); tiles flagged
// per CTA.
constexpr int TMA_EV_CAP = 1024;
constexpr int TMA_KFLAG_WORDS = 32;
template <int STAGES>
constexpr size_t tma_smem_bytes()
{
    return (size_t)STAGES * TMA_IN_STRIDE * 4 + 8 * STAGES + (size_t)TMA_EV_CAP * 12 + TMA_KFLAG_WORDS * 4 + 128;
}
// a stalled copy is given up after about two seconds at 2 GHz
constexpr long long TMA_WAIT_BUDGET = 4000000000ll;
static_assert(((TMA_IN_STRIDE * 4) % 128) == 0 && ((TMA_LX * 4) % 16) == 0, "smem alignment");
static_assert(2 * (tma_smem_bytes<2>() + 1024) <= 227 * 1024, "two CTAs per SM by shared memory");

constexpr int PLANE = TMA_LY * TMA_LX; // floats per staged plane

// Four consecutive staged values starting at p (16-byte aligned).
__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// The values a thread's four nodes pull for direction i: the staged row of
// the source, shifted by -ex_i. `b` points at the thread's first node in plane
// 0 (16-byte aligned).
template <int I>
__device__ __forceinline__ void pull4(const float *b, float v[4])
{
    const float *p = b + I * PLANE - ey(I) * TMA_LX;
    const float4 a = lds4(p);
    if constexpr (ex(I) == 0) {
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else if constexpr (ex(I) == 1) { // from x - 1
        v[0] = p[-1]; v[1] = a.x; v[2] = a.y; v[3] = a.z;
    } else {                           // from x + 1
        v[0] = a.y; v[1] = a.z; v[2] = a.w; v[3] = p[4];
    }
}

// The node's own populations of direction i (half-way bounce-back source).
template <int I>
__device__ __forceinline__ void own4(const float *b, float v[4])
{
    const float4 a = lds4(b + I * PLANE);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

// STAGES staged tiles per CTA, CTAS CTAs per SM (registers are capped so
// that they fit); NOISE: sigma != 0.
template <int STAGES, int CTAS, bool NOISE>
__global__ void __launch_bounds__(TMA_NT, CTAS)
    k_update_tma(SimDev d, int cur, uint32_t t, const __grid_constant__ CUtensorMap tm_in)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *s_in = (float *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint64_t *full = (uint64_t *)(s_in + STAGES * TMA_IN_STRIDE);
    // divisions of this CTA's tiles: local tile index, two staged offsets, amount
    int *ev_k = (int *)(full + STAGES);
    int *ev_off = ev_k + TMA_EV_CAP / 2;
    float *ev_add = (float *)(ev_off + TMA_EV_CAP);
    unsigned *kflag = (unsigned *)(ev_add + TMA_EV_CAP); // tiles with divisions
    __shared__ int s_abort, s_nev;

    const float *__restrict__ fin = (const float *)d.f[cur];
    float *__restrict__ fout = (float *)d.f[cur ^ 1];
    const int y_r = d.sc->y_r, y_copy = d.sc->y_copy, y_hi = d.sc->y_hi;
    const int W = d.W, H = d.H, Wp = d.Wp;
    const long long P = d.P;
    const int tid = threadIdx.x, lane = tid & 31, r = tid >> 5;

    // rows the rear wall has just frozen: bring this copy up to date
    if (y_copy < y_r) {
        const long long n = (long long)(y_r - y_copy) * Wp;
        for (long long k = (long long)blockIdx.x * TMA_NT + tid; k < n; k += (long long)gridDim.x * TMA_NT) {
            const long long o = (long long)y_copy * Wp + k;
#pragma unroll
            for (int i = 0; i < NQ; ++i) fout[i * P + o] = fin[i * P + o];
        }
    }

    const int ncx = (W + TMA_TX - 1) / TMA_TX;
    const int nrows = y_hi - y_r;
    const int nty = nrows > 0 ? (nrows + TMA_TY - 1) / TMA_TY : 0;
    const int ntiles = ncx * nty;
    const int G = (int)gridDim.x;
    const int count = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / G + 1 : 0;
    // tile k of this CTA is blockIdx.x + k G; its (tx, ty) advance by (G % ncx, G / ncx)
    const int dtx = G % ncx, dty = G / ncx;

    if (tid == 0) {
        s_abort = 0;
        s_nev = 0;
        prefetch_tensormap(&tm_in);
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    if (tid < TMA_KFLAG_WORDS) kflag[tid] = 0u;
    __syncthreads();
    int itx = (int)blockIdx.x % ncx, ity = (int)blockIdx.x / ncx; // next tile to load (thread 0)
    auto issue = [&](int k) {
        const int s = k % STAGES;
        mbar_arrive_expect_tx(&full[s], TMA_IN_BYTES);
        tma_load_3d(s_in + s * TMA_IN_STRIDE, &tm_in, itx * TMA_TX - 4, y_r + ity * TMA_TY - 1, 0, &full[s]);
        itx += dtx;
        ity += dty;
        if (itx >= ncx) {
            itx -= ncx;
            ++ity;
        }
    };
    // the first tiles' copies run while the divisions are sorted out below
    if (tid == 0)
        for (int k = 0; k < STAGES && k < count; ++k) issue(k);

    // App. A step 3 for this CTA: the selector listed, per division, the CTA
    // that owns its node's tile, the tile's local index, the offsets of the
    // two pre-stream slots in the staged box and the amount; keep ours.
    const int nev_all = d.inject_in_update ? d.sc->n_events : 0;
    constexpr int EV_BATCH = 16; // owner words a thread loads before it looks at any
    for (int eb = 0; eb < nev_all; eb += TMA_NT * EV_BATCH) {
        int own[EV_BATCH];
#pragma unroll
        for (int j = 0; j < EV_BATCH; ++j) {
            const int e = eb + j * TMA_NT + tid;
            own[j] = e < nev_all ? d.rec_owner[e] : -1;
        }
#pragma unroll
        for (int j = 0; j < EV_BATCH; ++j) {
            const int e = eb + j * TMA_NT + tid;
            if (own[j] == (int)blockIdx.x) {
                const int at = atomicAdd(&s_nev, 1);
                const int k = d.rec_k[e];
                if (at < TMA_EV_CAP / 2) {
                    ev_k[at] = k;
                    ev_off[2 * at] = d.rec_off[2 * e];
                    ev_off[2 * at + 1] = d.rec_off[2 * e + 1];
                    ev_add[at] = d.rec_add[e];
                }
                if (k < 32 * TMA_KFLAG_WORDS) atomicOr(&kflag[k >> 5], 1u << (k & 31));
            }
        }
    }
    __syncthreads();
    const int nev = s_nev;                            // divisions of this CTA
    const bool ev_overflow = nev > TMA_EV_CAP / 2;    // then scan the global list per tile

    const Consts<float> cf = make_consts<float>(d);
    const float rho_c = d.f_rho_c;
    // periodic wrap patch: thread (plane pq, staged row pyb) for tid < 9 LY
    const int pq = tid / TMA_LY, pyb = tid - pq * TMA_LY;
    const bool patcher = tid < 9 * TMA_LY;
    long long mass = 0;
    int maxrow = -1;
    float clip = 0.0f;
    int done = 0;
    int tx = (int)blockIdx.x % ncx, ty = (int)blockIdx.x / ncx;

    for (int k = 0; k < count; ++k) {
        const int s = k % STAGES;
        const uint32_t parity = (uint32_t)((k / STAGES) & 1);
        const int x0 = tx * TMA_TX, y0 = y_r + ty * TMA_TY;
        float *stage = s_in + s * TMA_IN_STRIDE;
        // periodic wrap: the staged column x = -1 holds x = W - 1 and the
        // column x = W holds x = 0
        const bool left = tx == 0, right = tx == ncx - 1;
        const int pyg = y0 - 1 + pyb;
        const bool pok = patcher && (left || right) && pyg >= 0 && pyg < H;
        float pl = 0.0f, pr = 0.0f;
        if (pok) {
            const float *rowp = fin + pq * P + (long long)pyg * Wp;
            if (left) pl = rowp[W - 1];
            if (right) pr = rowp[0];
        }
        if (!mbar_wait_bounded(&full[s], parity, TMA_WAIT_BUDGET)) atomicOr(&s_abort, 1);
        if (left || right) { // uniform across the CTA
            if (pok) {
                float *sp = stage + pq * PLANE + pyb * TMA_LX;
                if (left) sp[3] = pl;
                if (right) sp[(W - x0) + 4] = pr;
                fence_proxy_async_smem(); // before the next bulk copy overwrites them
            }
            __syncthreads();
        }
        // divisions of this tile, added to the staged pre-stream slots
        const bool has_ev = nev > 0 && (ev_overflow || k >= 32 * TMA_KFLAG_WORDS || ((kflag[k >> 5] >> (k & 31)) & 1u));
        if (has_ev) { // uniform across the CTA
            if (!ev_overflow) {
                for (int i = tid; i < nev; i += TMA_NT)
                    if (ev_k[i] == k) {
                        stage[ev_off[2 * i]] += ev_add[i];
                        stage[ev_off[2 * i + 1]] += ev_add[i];
                    }
            } else {
                for (int e = tid; e < nev_all; e += TMA_NT)
                    if (d.rec_owner[e] == (int)blockIdx.x && d.rec_k[e] == k) {
                        stage[d.rec_off[2 * e]] += d.rec_add[e];
                        stage[d.rec_off[2 * e + 1]] += d.rec_add[e];
                    }
            }
            fence_proxy_async_smem();
            __syncthreads();
        }
        if (s_abort) break;
        const int y = y0 + r;
        const bool active = y < y_hi; // rows past the active window hold no mass (warp-uniform)
        const int xb = x0 + 4 * lane;  // first of this thread's four columns
        float g[NQ][4];
        if (active) {
            const float *b = stage + (r + 1) * TMA_LX + 4 * lane + 4;
            pull4<0>(b, g[0]);
            pull4<1>(b, g[1]);
            pull4<3>(b, g[3]);
            if (y - 1 < y_r) { // rear wall: half-way bounce-back
                own4<4>(b, g[2]);
                own4<7>(b, g[5]);
                own4<8>(b, g[6]);
            } else {
                pull4<2>(b, g[2]);
                pull4<5>(b, g[5]);
                pull4<6>(b, g[6]);
            }
            if (y + 1 >= H) { // top wall
                own4<2>(b, g[4]);
                own4<5>(b, g[7]);
                own4<6>(b, g[8]);
            } else {
                pull4<4>(b, g[4]);
                pull4<7>(b, g[7]);
                pull4<8>(b, g[8]);
            }
        }
        __syncthreads(); // the tile is in registers: the stage is free
        if (tid == 0 && k + STAGES < count) issue(k + STAGES);
        if (active) {
            float fo[NQ][4];
            float rho[4], added[4];
            bool occ[4];
            unsigned nib = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float r0 = g[0][j];
#pragma unroll
                for (int i = 1; i < NQ; ++i) r0 = r0 + g[i][j];
                rho[j] = r0;
                occ[j] = xb + j < W && r0 >= rho_c;
                added[j] = 0.0f;
                nib |= (unsigned)occ[j] << j;
            }
            if (__all_sync(0xffffffffu, nib == 15u)) {
                // the bulk: every node of the warp's row is occupied
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float gj[NQ], fj[NQ];
#pragma unroll
                    for (int i = 0; i < NQ; ++i) gj[i] = g[i][j];
                    relax_core<float, NOISE>(gj, rho[j], fj, (uint32_t)(y * W + xb + j), t, d, cf);
#pragma unroll
                    for (int i = 0; i < NQ; ++i) fo[i][j] = fj[i];
                }
                float mn = fo[0][0];
#pragma unroll
                for (int i = 0; i < NQ; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) mn = fminf(mn, fo[i][j]);
                if (__any_sync(0xffffffffu, mn < 0.0f)) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float fj[NQ];
#pragma unroll
                        for (int i = 0; i < NQ; ++i) fj[i] = fo[i][j];
                        added[j] = fix_negative<float>(fj, d.negfix);
#pragma unroll
                        for (int i = 0; i < NQ; ++i) fo[i][j] = fj[i];
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float gj[NQ], fj[NQ];
#pragma unroll
                    for (int i = 0; i < NQ; ++i) gj[i] = g[i][j];
                    if (occ[j]) {
                        relax_core<float, NOISE>(gj, rho[j], fj, (uint32_t)(y * W + xb + j), t, d, cf);
                        added[j] = fix_negative<float>(fj, d.negfix);
                    } else {
#pragma unroll
                        for (int i = 0; i < NQ; ++i) fj[i] = gj[opp(i)];
                    }
#pragma unroll
                    for (int i = 0; i < NQ; ++i) fo[i][j] = fj[i];
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (xb + j < W) {
                    clip += added[j];
                    float fj[NQ];
#pragma unroll
                    for (int i = 0; i < NQ; ++i) fj[i] = fo[i][j];
                    const float ro = node_mass<float>(fj, rho[j], added[j]);
                    mass += fix24<float>(ro);
                    if (ro != 0.0f) maxrow = y;
                }
            }
            // occupancy bits: lanes 8m..8m+7 hold the 32 columns of word m
            unsigned v = nib << (4 * (lane & 7));
            v |= __shfl_xor_sync(0xffffffffu, v, 1);
            v |= __shfl_xor_sync(0xffffffffu, v, 2);
            v |= __shfl_xor_sync(0xffffffffu, v, 4);
            const int wx = (x0 >> 5) + (lane >> 3);
            if ((lane & 7) == 0 && wx < d.MW) d.mask[(long long)y * d.MW + wx] = v;
            // four columns at a time; columns in [W, Wp) are padding nobody reads
            if (xb < Wp) {
                float *o = fout + (long long)y * Wp + xb;
#pragma unroll
                for (int i = 0; i < NQ; ++i)
                    *reinterpret_cast<float4 *>(o + i * P) = make_float4(fo[i][0], fo[i][1], fo[i][2], fo[i][3]);
            }
        }
        tx += dtx;
        ty += dty;
        if (tx >= ncx) {
            tx -= ncx;
            ++ty;
        }
        ++done;
    }
    if (tid == 0 && s_abort) {
        atomicOr(&d.sc->status, ST_TIMEOUT);
        // let every copy this CTA issued land before the CTA exits
        for (int k = done; k < count && k < done + STAGES; ++k)
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

template <int STAGES, int CTAS, bool NOISE>
cudaError_t launch_update_tma_variant(const SimDev &d, int cur, uint32_t t, const CUtensorMap *maps, int nsm,
                                      cudaStream_t s)
{
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !attr[dev]) {
        e = cudaFuncSetAttribute(k_update_tma<STAGES, CTAS, NOISE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tma_smem_bytes<STAGES>());
        if (e != cudaSuccess) return e;
        if (dev < 64) attr[dev] = true;
    }
    // maps[b] loads from population copy b
    k_update_tma<STAGES, CTAS, NOISE><<<CTAS * nsm, TMA_NT, tma_smem_bytes<STAGES>(), s>>>(d, cur, t, maps[cur]);
    return cudaGetLastError();
}

// variant 0: two staged tiles, two CTAs per SM; variant 1: one staged tile,
// three CTAs per SM
inline cudaError_t launch_update_tma(const SimDev &d, int cur, uint32_t t, const CUtensorMap *maps, int nsm,
                                     int variant, cudaStream_t s)
{
    if (variant == 1)
        return d.noise_on ? launch_update_tma_variant<1, 3, true>(d, cur, t, maps, nsm, s)
                          : launch_update_tma_variant<1, 3, false>(d, cur, t, maps, nsm, s);
    return d.noise_on ? launch_update_tma_variant<2, 2, true>(d, cur, t, maps, nsm, s)
                      : launch_update_tma_variant<2, 2, false>(d, cur, t, maps, nsm, s);
}

} // namespace lbm
