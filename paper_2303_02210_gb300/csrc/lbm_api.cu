// C ABI of the library (declared in include/lbm.h): parameter checks, device
// memory layout, initial front profile, launch sequencing and read-back.
// All lattice arithmetic runs in the kernels of lbm_kernels.cuh; the host only
// computes the initial front profile (App. A, first paragraph) and marshals.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <thread>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/lbm.h"
#include "lbm_common.cuh"
#include "lbm_tuned.h"

using namespace lbm;

namespace {

thread_local char g_cuda_err[256] = "no CUDA error";

int cuda_fail(cudaError_t e)
{
    std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return LBM_ERR_OOM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver || e == cudaErrorNoKernelImageForDevice)
        return LBM_ERR_NO_DEVICE;
    return LBM_ERR_CUDA;
}

// Every call on a handle makes the handle's device current first.
#define USE_DEVICE(s)                                                                                                  \
    do {                                                                                                               \
        cudaError_t e_ = cudaSetDevice((s)->device);                                                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_);                                                                   \
    } while (0)

#define CK(call)                                                                                                       \
    do {                                                                                                               \
        cudaError_t e_ = (call);                                                                                       \
        if (e_ != cudaSuccess) return cuda_fail(e_);                                                                   \
    } while (0)

uint64_t align256(uint64_t v) { return (v + 255u) & ~uint64_t(255u); }

// The tuned entry for a storage type and width: the largest tuned width not
// above W (the smallest tuned width if all are); nullptr if the table has no
// entry for the storage type.
const TunedShape *tuned_shape(int precision, int width)
{
    const TunedShape *best = nullptr, *least = nullptr;
    for (int i = 0; i < kTunedShapeCount; ++i) {
        const TunedShape &t = kTunedShapes[i];
        if (t.precision != precision) continue;
        if (!least || t.width < least->width) least = &t;
        if (t.width <= width && (!best || t.width > best->width)) best = &t;
    }
    return best ? best : least;
}

// The kernels of a lattice and storage type.
const KernelTable *kernel_table(int lattice, int precision)
{
    if (lattice == LBM_D2Q7) return precision == LBM_FP64 ? &kTableF64Q7 : &kTableF32Q7;
    return precision == LBM_FP64   ? &kTableF64
           : precision == LBM_FP16 ? &kTableF16
           : precision == LBM_BF16 ? &kTableBF16
                                   : &kTableF32;
}

// 16-bit population storage on the host side: the shift c_k = w_k rho_init
// rounded to the storage type (weight class k: 0 rest, 1 axis, 2 diagonal),
// and the same decode (float(s) + c, in FP32) and encode (round f - c to
// nearest) as the kernels.
float pop_shift(int precision, int k, double rho_init)
{
    const double w = k == 0 ? 4.0 / 9.0 : (k == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    const float c = (float)(w * rho_init);
    if (precision == LBM_FP16) return __half2float(__float2half_rn(c));
    if (precision == LBM_BF16) return __bfloat162float(__float2bfloat16_rn(c));
    return 0.0f;
}
int plane_class(int i) { return i == 0 ? 0 : (i < 5 ? 1 : 2); }
double decode16(int precision, uint16_t bits, float c)
{
    float v;
    if (precision == LBM_FP16) {
        __half h;
        std::memcpy(&h, &bits, 2);
        v = __half2float(h);
    } else {
        __nv_bfloat16 h;
        std::memcpy(&h, &bits, 2);
        v = __bfloat162float(h);
    }
    return (double)(v + c);
}
uint16_t encode16(int precision, double f, float c)
{
    const float v = (float)f - c;
    uint16_t bits;
    if (precision == LBM_FP16) {
        const __half h = __float2half_rn(v);
        std::memcpy(&bits, &h, 2);
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        std::memcpy(&bits, &h, 2);
    }
    return bits;
}

struct Layout {
    int Wp, MW, hcap, ns_max;
    int Q; // lattice directions (population planes)
    long long P;
    int elem;
    uint64_t off_f0, off_f1, off_mask, off_heights, off_rows0, off_sc, off_htab, off_hlist, off_evk,
        off_evc, off_rown, off_rk, off_roff, off_bcnt, off_bucket, off_pl64, off_pl32, total;
};

Layout make_layout(const lbm_params_t &p)
{
    Layout L{};
    L.elem = p.precision == LBM_FP64 ? 8 : (p.precision == LBM_FP32 ? 4 : 2);
    L.Q = p.lattice == LBM_D2Q7 ? 7 : 9;
    // stored row: kXO columns left of x = 0 (x = -1 the ghost of W - 1), the
    // W columns, the ghost of column 0 at x = W, padding to 128 bytes of FP32
    L.Wp = (p.width + 2 * kXO + 31) / 32 * 32;
    L.MW = (p.width + 31) / 32;
    L.P = (long long)L.Wp * p.height;
    // planner capacity: divisions per step at up to four times the initial
    // density over the whole lattice, at least 1024
    double est = 0.0;
    if (p.growth_mode != LBM_GROW_NONE) {
        const double rho_hi = 4.0 * std::max(p.rho_init * (1.0 + std::fabs(p.rho_jitter)), p.rho_c);
        est = p.growth_rate * rho_hi * (double)p.width * (double)p.height / p.rho_cell;
    }
    double cap = std::ceil(est) + 1024.0;
    if (cap > 16777216.0) cap = 16777216.0;
    L.ns_max = (int)cap;
    L.hcap = 1;
    while (L.hcap < 2 * L.ns_max) L.hcap <<= 1;
    uint64_t o = 0;
    const uint64_t fbytes = (uint64_t)L.Q * (uint64_t)L.P * (uint64_t)L.elem;
    L.off_f0 = o; o = align256(o + fbytes);
    L.off_f1 = o; o = align256(o + fbytes);
    L.off_mask = o; o = align256(o + (uint64_t)p.height * L.MW * 4u);
    L.off_heights = o; o = align256(o + (uint64_t)p.width * 4u);
    L.off_rows0 = o; o = align256(o + (uint64_t)p.width * 4u);
    L.off_sc = o; o = align256(o + sizeof(DevScalars));
    L.off_htab = o; o = align256(o + (uint64_t)L.hcap * 8u);
    L.off_hlist = o; o = align256(o + (uint64_t)L.ns_max * 4u);
    // event lists of two consecutive steps (the planner selects one step ahead)
    L.off_evk = o; o = align256(o + (uint64_t)L.ns_max * 8u);
    L.off_evc = o; o = align256(o + (uint64_t)L.ns_max * 8u);
    L.off_rown = o; o = align256(o + (uint64_t)L.ns_max * 4u);
    L.off_rk = o; o = align256(o + (uint64_t)L.ns_max * 4u);
    L.off_roff = o; o = align256(o + (uint64_t)L.ns_max * 8u);
    L.off_bcnt = o; o = align256(o + (uint64_t)kTmaMaxCtas * 4u);
    L.off_bucket = o; o = align256(o + (uint64_t)kTmaMaxCtas * kBucketCap * 4u);
    // planner partials: S1, S2, frozen mass (int64); top, low, two count buffers (int32)
    L.off_pl64 = o; o = align256(o + (uint64_t)kPlanMaxBlocks * 3u * 8u);
    L.off_pl32 = o; o = align256(o + (uint64_t)kPlanMaxBlocks * 4u * 4u);
    L.total = o;
    return L;
}

// Initial front (App. A: a flat interface; here optionally perturbed): the
// number of tissue rows of each column, node (x, y) being tissue iff y < h0(x).
void front_rows(const lbm_params_t &p, std::vector<int32_t> &rows)
{
    const int W = p.width, H = p.height;
    const PhiloxKey pk = philox_key((uint32_t)(p.seed & 0xFFFFFFFFu), (uint32_t)(p.seed >> 32));
    rows.assign(W, H);
    if (p.front_kind == LBM_FRONT_FULL) return;
    std::vector<double> h0(W);
    if (p.front_kind == LBM_FRONT_FLAT) {
        for (int x = 0; x < W; ++x) {
            const u32x4 r = philox4x32_10(u32x4{(uint32_t)x, 0u, STREAM_INIT, p.sim_id}, pk);
            h0[x] = p.front_row + p.front_amp * (2.0 * u01(r.x) - 1.0);
        }
    } else {
        // sum of sinusoids k = kmin..kmax with phases 2 pi U_k, scaled so that
        // its largest excursion equals the amplitude
        const double two_pi = 6.283185307179586;
        std::vector<double> phi;
        for (int k = p.front_kmin; k <= p.front_kmax; ++k) {
            const u32x4 r = philox4x32_10(u32x4{(uint32_t)k, 1u, STREAM_INIT, p.sim_id}, pk);
            phi.push_back(two_pi * u01(r.x));
        }
        // each column's sum in the same order whatever thread forms it (so
        // the values do not depend on the split); columns split over host
        // threads when the sum is long (4096 columns x 64 modes: ~4 ms on one
        // core, inside every lbm_create of the benchmark workload)
        auto columns = [&](int x0, int x1) {
            for (int x = x0; x < x1; ++x) {
                double S = 0.0;
                for (int k = p.front_kmin; k <= p.front_kmax; ++k)
                    S = S + std::sin(((two_pi * (double)k) * (double)x) / (double)W + phi[k - p.front_kmin]);
                h0[x] = S;
            }
        };
        const long long work = (long long)W * (long long)phi.size();
        const int nt = (int)std::min<long long>({(long long)std::max(1u, std::thread::hardware_concurrency()), 16LL,
                                                 work / 16384 + 1});
        if (nt <= 1) {
            columns(0, W);
        } else {
            std::vector<std::thread> pool;
            for (int i = 1; i < nt; ++i) pool.emplace_back(columns, (int)((long long)W * i / nt), (int)((long long)W * (i + 1) / nt));
            columns(0, (int)((long long)W / nt));
            for (std::thread &t : pool) t.join();
        }
        double smax = 0.0;
        for (int x = 0; x < W; ++x)
            if (std::fabs(h0[x]) > smax) smax = std::fabs(h0[x]);
        for (int x = 0; x < W; ++x)
            h0[x] = smax > 0.0 ? p.front_row + p.front_amp * (h0[x] / smax) : p.front_row;
    }
    for (int x = 0; x < W; ++x) {
        double c = std::ceil(h0[x]);
        if (c < 0.0) c = 0.0;
        if (c > (double)H) c = (double)H;
        rows[x] = (int32_t)c;
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link-time dependency on the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// Population copy as a 3-D tensor {nx, H, Q} of stored rows (coordinate
// x_stored = x + kXO, so the ghost columns are inside when nx = Wp) with row
// pitch Wp and plane pitch P elements; `bx` x `by` x Q boxes. Out-of-range
// loads read zeros; stores are cut at the tensor's edges (nx = W + kXO cuts
// them at x = W - 1).
bool encode_population_map(CUtensorMap *m, void *base, int nx, int Wp, int H, long long P, int Q, int bx, int by,
                           int precision)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t el = precision == LBM_FP32 ? 4u : 2u;
    const CUtensorMapDataType dt = precision == LBM_FP32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : precision == LBM_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                           : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)H, (cuuint64_t)Q};
    const cuuint64_t strides[2] = {(cuuint64_t)Wp * el, (cuuint64_t)P * el};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)Q};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

} // namespace

int lbm::lbm_record_cuda_error(cudaError_t e) { return cuda_fail(e); }

struct lbm_sim {
    lbm_params_t p;
    int device;
    SimDev d;
    Layout L;
    const KernelTable *kt;
    cudaStream_t stream;
    void *arena;
    bool own_arena;
    int cur;
    int64_t step;
    int64_t launches;
    // TMA-staged update (FP32, walls in y)
    bool use_tma;
    int tma_grid, tma_variant;
    CUtensorMap maps[4]; // loads from copy 0, 1; stores into copy 0, 1 (variants that store in bulk)
    // kernel timing
    std::vector<cudaEvent_t> ev;
    int64_t ev_used;
    bool timing;
    int64_t timing_nodes0;
    int64_t timing_stride, timing_count;
};

namespace {
// Copies the front heights (W int32) and the two Eq. 6 sums into host memory
// that the device can address (pinned, mapped), by stores from the GPU: one
// small launch in place of two copy-engine transfers, each of which would
// stall the stream for several microseconds between two steps.
// Launched as a programmatic dependent of the planner: it may start while the
// planner finishes and waits for it before reading.
__global__ void k_export_front(const int32_t *__restrict__ h, const long long *__restrict__ s12, int W,
                               int32_t *h_out, long long *s_out)
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); // (the next update may start its prologue)
    asm volatile("griddepcontrol.wait;" ::: "memory");               // what the planner wrote
    const int stride = (int)(gridDim.x * blockDim.x);
    if (h_out)
        for (int i = (int)(blockIdx.x * blockDim.x + threadIdx.x); i < W; i += stride) h_out[i] = h[i];
    if (blockIdx.x == 0 && threadIdx.x < 2) s_out[threadIdx.x] = s12[threadIdx.x];
}

// The device's address of host memory p, or nullptr if the current device
// cannot address it (pageable memory, or pinned memory not mapped for it).
void *device_alias(void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError(); // (pageable memory may leave an error on older runtimes)
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}
} // namespace

extern "C" {

int lbm_validate(const lbm_params_t *p)
{
    if (!p) return LBM_ERR_INVALID_ARG;
    if (p->width < 1 || p->height < 3 || p->width > 32768 || p->height > 32768) return LBM_ERR_INVALID_ARG;
    if ((int64_t)p->width * p->height >= (int64_t)1 << 30) return LBM_ERR_INVALID_ARG;
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return LBM_ERR_INVALID_ARG;
    if (!(p->rho_cell > 0.0) || !(p->rho_c >= 0.0) || !(p->growth_rate >= 0.0) || !(p->sigma >= 0.0))
        return LBM_ERR_INVALID_ARG;
    if (!std::isfinite(p->mu) || !std::isfinite(p->rho_init) || !(p->rho_init >= 0.0)) return LBM_ERR_INVALID_ARG;
    if (p->growth_mode < LBM_GROW_NONE || p->growth_mode > LBM_GROW_BAND) return LBM_ERR_INVALID_ARG;
    if (p->growth_mode == LBM_GROW_DENSITY && !(p->rho0 > 0.0)) return LBM_ERR_INVALID_ARG;
    if (p->growth_mode == LBM_GROW_EDGE && p->edge_depth < 0) return LBM_ERR_INVALID_ARG;
    if (p->growth_mode == LBM_GROW_BAND && p->band_rows < 1) return LBM_ERR_INVALID_ARG;
    if (p->front_kind < LBM_FRONT_FLAT || p->front_kind > LBM_FRONT_FULL) return LBM_ERR_INVALID_ARG;
    if (p->front_kind == LBM_FRONT_SINUSOIDAL && (p->front_kmin < 0 || p->front_kmax < p->front_kmin))
        return LBM_ERR_INVALID_ARG;
    if (p->wall_mode != LBM_WALL_FIXED && p->wall_mode != LBM_WALL_ADVANCE) return LBM_ERR_INVALID_ARG;
    if (p->negfix_mode != LBM_NEGFIX_LITERAL && p->negfix_mode != LBM_NEGFIX_RESCALE) return LBM_ERR_INVALID_ARG;
    if (p->precision < LBM_FP32 || p->precision > LBM_BF16) return LBM_ERR_INVALID_ARG;
    if (p->y_periodic != 0 && p->y_periodic != 1) return LBM_ERR_INVALID_ARG;
    if (p->update_kernel < 0 || p->update_kernel > 6) return LBM_ERR_INVALID_ARG;
    if (p->plan_blocks < 0 || p->plan_blocks > kPlanMaxBlocks) return LBM_ERR_INVALID_ARG;
    if (p->update_kernel >= 2 && p->update_kernel != 5 && (p->precision == LBM_FP64 || p->y_periodic))
        return LBM_ERR_INVALID_ARG;
    // bulk tensor stores: FP32 only (16-bit tiles start off a 16-byte boundary)
    if (p->update_kernel == 6 && p->precision != LBM_FP32) return LBM_ERR_INVALID_ARG;
    if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D2Q7) return LBM_ERR_INVALID_ARG;
    // D2Q7: FP32 or FP64 storage, the plain-load or the (one) TMA-staged
    // update, an even H when periodic in y
    if (p->lattice == LBM_D2Q7 &&
        ((p->precision != LBM_FP32 && p->precision != LBM_FP64) || p->update_kernel == 3 || p->update_kernel == 4 ||
         p->update_kernel == 6 || (p->y_periodic && (p->height & 1))))
        return LBM_ERR_INVALID_ARG;
    return LBM_OK;
}

int lbm_plan_capacity(const lbm_params_t *p, int64_t *ns_max)
{
    if (!ns_max) return LBM_ERR_INVALID_ARG;
    const int v = lbm_validate(p);
    if (v != LBM_OK) return v;
    *ns_max = make_layout(*p).ns_max;
    return LBM_OK;
}

int lbm_footprint(const lbm_params_t *p, uint64_t *bytes)
{
    if (!bytes) return LBM_ERR_INVALID_ARG;
    const int v = lbm_validate(p);
    if (v != LBM_OK) return v;
    *bytes = make_layout(*p).total;
    return LBM_OK;
}

void lbm_destroy(lbm_sim *s)
{
    if (!s) return;
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->stream);
    for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
    if (s->own_arena && s->arena) cudaFree(s->arena);
    delete s;
}

int lbm_create(const lbm_params_t *p, void *stream, void *arena, uint64_t arena_bytes, lbm_sim **out)
{
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    int v = lbm_validate(p);
    if (v != LBM_OK) return v;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));

    lbm_sim *s = new lbm_sim();
    s->p = *p;
    s->device = dev;
    s->L = make_layout(*p);
    s->kt = kernel_table(p->lattice, p->precision);
    s->stream = (cudaStream_t)stream;
    s->cur = 0;
    s->step = 0;
    s->launches = 0;
    s->ev_used = 0;
    s->timing = false;
    s->timing_stride = 1;
    s->timing_count = 0;
    if (arena) {
        if (arena_bytes < s->L.total || ((uintptr_t)arena & 255u) != 0) {
            delete s;
            return arena_bytes < s->L.total ? LBM_ERR_OOM : LBM_ERR_INVALID_ARG;
        }
        s->arena = arena;
        s->own_arena = false;
    } else {
        cudaError_t e = cudaMalloc(&s->arena, s->L.total);
        if (e != cudaSuccess) {
            delete s;
            return cuda_fail(e);
        }
        s->own_arena = true;
    }
    char *base = (char *)s->arena;
    const Layout &L = s->L;
    SimDev &d = s->d;
    std::memset(&d, 0, sizeof(d));
    d.f[0] = base + L.off_f0 + (size_t)kXO * L.elem;
    d.f[1] = base + L.off_f1 + (size_t)kXO * L.elem;
    d.mask = (uint32_t *)(base + L.off_mask);
    d.heights = (int32_t *)(base + L.off_heights);
    d.rows0 = (int32_t *)(base + L.off_rows0);
    d.sc = (DevScalars *)(base + L.off_sc);
    d.htab = (unsigned long long *)(base + L.off_htab);
    d.hlist = (int32_t *)(base + L.off_hlist);
    d.ev_key = (uint32_t *)(base + L.off_evk);
    d.ev_count = (int32_t *)(base + L.off_evc);
    d.rec_owner = (int *)(base + L.off_rown);
    d.rec_k = (int *)(base + L.off_rk);
    d.rec_off = (int *)(base + L.off_roff);
    d.bucket_cnt = (int *)(base + L.off_bcnt);
    d.bucket = (int *)(base + L.off_bucket);
    d.pl_s1 = (long long *)(base + L.off_pl64);
    d.pl_s2 = d.pl_s1 + kPlanMaxBlocks;
    d.pl_mass = d.pl_s2 + kPlanMaxBlocks;
    d.pl_top = (int *)(base + L.off_pl32);
    d.pl_low = d.pl_top + kPlanMaxBlocks;
    d.pl_cnt = d.pl_low + kPlanMaxBlocks; // two buffers
    d.W = p->width;
    d.H = p->height;
    d.Wp = L.Wp;
    d.MW = L.MW;
    d.P = L.P;
    d.hcap = L.hcap;
    d.ns_max = L.ns_max;
    d.omega = 1.0 / p->tau;
    d.cmu = 1.0 - p->mu;
    d.rho_c = p->rho_c;
    d.rho_cell = p->rho_cell;
    d.half_cell = p->rho_cell * 0.5;
    d.growth_rate = p->growth_rate;
    d.rho0 = p->rho0;
    d.sigma = p->sigma;
    d.rho_init = p->rho_init;
    d.rho_jitter = p->rho_jitter;
    d.wall_min_gap = p->wall_min_gap;
    d.wall_w_factor = p->wall_w_factor;
    d.key0 = (uint32_t)(p->seed & 0xFFFFFFFFu);
    d.key1 = (uint32_t)(p->seed >> 32);
    d.pk = philox_key(d.key0, d.key1);
    d.sim = p->sim_id;
    d.growth_mode = p->growth_mode;
    d.edge_depth = p->edge_depth;
    d.band_rows = p->band_rows;
    d.wall_mode = p->wall_mode;
    d.negfix = p->negfix_mode;
    d.y_periodic = p->y_periodic;
    d.noise_on = p->sigma != 0.0;
    d.f_rho_c = (float)d.rho_c;
    d.f_omega = (float)d.omega;
    d.f_cmu = (float)d.cmu;
    d.f_om1 = (float)(1.0 - d.omega);
    d.f_ow0 = (float)(d.omega * (4.0 / 9.0));
    d.f_ow1 = (float)(d.omega * (1.0 / 9.0));
    d.f_ow5 = (float)(d.omega * (1.0 / 36.0));
    d.f_two_sigma = (float)(2.0 * p->sigma);
    for (int k = 0; k < 3; ++k) d.pop_shift[k] = pop_shift(p->precision, k, p->rho_init);
    const int bps = s->kt->update_blocks_per_sm();
    // persistent grid: as many blocks as fit on the SMs, rounded down to a
    // multiple of the column tiles (each block keeps one column tile)
    const int ncx = (p->width + s->kt->update_tile_x - 1) / s->kt->update_tile_x;
    const int g0 = nsm * (bps > 0 ? bps : 1);
    d.update_grid = g0 >= ncx ? (g0 / ncx) * ncx : ncx;
    // the planner's blocks must all be resident at once (cooperative launch)
    const int pbs = s->kt->plan_blocks_per_sm(0);
    // one 32-column mask word per warp, about one candidate per thread at
    // the largest n_s; at least two blocks, at most a quarter of the SMs
    // (every grid barrier costs an arrival per block; measured on the edge-
    // growth workload with 17, 34, 38 and 48 blocks, the FP32 step took 77.9,
    // 76.6, 76.3 and 77.4 us at 4096 x 2048 and 147.6, 143.1, 142.8 and
    // 142.4 us at 8192 x 2048)
    const long long want = std::max<long long>((L.MW + 15) / 16, (L.ns_max + 511) / 512);
    int pg = (int)std::min<long long>(std::max(2, nsm / 4), std::max<long long>(2, want));
    // the tuned table's grid for this storage type and width (D2Q9), or the
    // caller's; at most the resident count
    const TunedShape *tuned = p->lattice == LBM_D2Q9 ? tuned_shape(p->precision, p->width) : nullptr;
    if (p->plan_blocks > 0) {
        if (p->plan_blocks > pbs * nsm) {
            if (s->own_arena) cudaFree(s->arena);
            delete s;
            return LBM_ERR_INVALID_ARG;
        }
        pg = p->plan_blocks;
    } else if (tuned && tuned->plan_blocks > 0) {
        pg = std::min(tuned->plan_blocks, pbs * nsm);
    }
    d.plan_grid = pbs > 0 ? std::min(pg, kPlanMaxBlocks) : 0;
    if (d.plan_grid < 1) {
        if (s->own_arena) cudaFree(s->arena);
        delete s;
        return LBM_ERR_CUDA;
    }
    s->use_tma = false;
    s->tma_grid = nsm;
    // staged update variant (KernelTable::tma_info): "tma" 0 (two-row tiles),
    // "tma1" 1 (four-row tiles), "tma_st" 2 (two-row tiles stored in bulk,
    // FP32). Automatic: the tuned table's form for the storage type and
    // width (lbm_tuned.h, written by the autotuner's sweep); without an entry
    // the hand-set rule: the bulk-store form for FP32 from 2048 columns on
    // (measured per update launch: 57.3 against 62.7 us at 4096 x 2048, 115
    // against 124 (four-row tiles) at 8192 x 2048, 32.7 against 33.9 at
    // 2048), two-row tiles below (19.1 against 21.1 us at 1024, where the
    // window stays in the L2) and for 16-bit storage up to 4096 columns,
    // four-row tiles beyond. The four-row form for a simulation that shares
    // the GPU (5: 15.1 against 12.5 G node updates/s aggregate for a hundred
    // concurrent requests). D2Q7: one form.
    // The bulk-store form cuts its stores at x = W - 1, and a bulk store
    // writes the 16-byte unit that holds its last column whole: with W + 4
    // not a multiple of 4 elements that would overwrite the ghost column
    // x = W, so such widths keep the per-lane stores.
    const bool bulk_ok = p->precision == LBM_FP32 && p->width % 4 == 0;
    int variant = 0;
    if (p->lattice == LBM_D2Q9) {
        if (p->update_kernel == 3 || p->update_kernel == 5)
            variant = 1;
        else if (p->update_kernel == 6)
            variant = bulk_ok ? 2 : 0;
        else if (p->update_kernel == 0) {
            variant = tuned ? tuned->variant : (bulk_ok && p->width >= 2048 ? 2 : (p->width > 4096 ? 1 : 0));
            if (variant == 2 && !bulk_ok) variant = 0;
        }
    }
    s->tma_variant = variant;
    const bool tma_inject = p->update_kernel != 4; // 4: the selector injects into global memory
    int box_rows = 0, iter_rows = 0, ctas_per_sm = 0;
    const int kind = s->kt->tma_info ? s->kt->tma_info(variant, &box_rows, &iter_rows, &ctas_per_sm) : -1;
    if (kind >= 0 && s->kt->tma_update && !p->y_periodic && p->update_kernel != 1) {
        bool ok = true;
        for (int b = 0; b < 2 && ok; ++b)
            ok = encode_population_map(&s->maps[b], (char *)d.f[b] - (size_t)kXO * L.elem, d.Wp, d.Wp, d.H, d.P, L.Q,
                                       kTmaBoxX + 8, box_rows, p->precision);
        // bulk stores of a tile's 128 columns, cut at x = W - 1 (the ghost
        // columns are written by the edge lanes)
        for (int b = 0; b < 2 && ok && kind == 1; ++b)
            ok = encode_population_map(&s->maps[2 + b], (char *)d.f[b] - (size_t)kXO * L.elem, p->width + kXO, d.Wp,
                                       d.H, d.P, L.Q, kTmaBoxX, iter_rows, p->precision);
        s->use_tma = ok;
        d.inject_in_update = ok && tma_inject ? 1 : 0;
        const int ty = iter_rows;
        d.upd_tyl2 = 0;
        while ((1 << d.upd_tyl2) < ty) ++d.upd_tyl2;
        // persistent CTAs, but no more than one per eight tiles of the whole
        // lattice (small lattices then leave SMs to others in a batch); at
        // least two, since the reciprocal below needs upd_ctas >= 2
        const long long tiles = (long long)((p->width + kTmaBoxX - 1) / kTmaBoxX) * ((p->height + ty - 1) / ty);
        d.upd_ctas = (int)std::max<long long>(2, std::min<long long>((long long)ctas_per_sm * nsm, (tiles + 7) / 8));
        d.upd_magic = (uint32_t)((((uint64_t)1 << 32) + (uint64_t)d.upd_ctas - 1) / (uint64_t)d.upd_ctas);
        // (tile / upd_ctas by the reciprocal is exact while tile * upd_ctas < 2^32)
        if (d.upd_ctas > kTmaMaxCtas || tiles * (long long)d.upd_ctas >= (1LL << 32)) {
            s->use_tma = false;
            d.inject_in_update = 0;
        }
        if (!ok && p->update_kernel >= 2 && p->update_kernel != 5) {
            if (s->own_arena) cudaFree(s->arena);
            delete s;
            return LBM_ERR_CUDA;
        }
    }

    int rc = LBM_OK;
    do {
        cudaError_t e = cudaMemsetAsync(s->arena, 0, L.total, s->stream);
        if (e != cudaSuccess) { rc = cuda_fail(e); break; }
        // the division table starts empty (every entry all ones)
        e = cudaMemsetAsync(d.htab, 0xFF, (size_t)L.hcap * 8u, s->stream);
        if (e != cudaSuccess) { rc = cuda_fail(e); break; }
        std::vector<int32_t> rows;
        front_rows(*p, rows);
        e = cudaMemcpyAsync(d.rows0, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) { rc = cuda_fail(e); break; }
        if ((e = s->kt->fill(d, s->stream)) != cudaSuccess) { rc = cuda_fail(e); break; }
        if ((e = s->kt->scan(d, 0, s->stream)) != cudaSuccess) { rc = cuda_fail(e); break; }
        // observables of the initial state and the divisions of step 0
        if ((e = s->kt->plan(d, 1, s->stream)) != cudaSuccess) { rc = cuda_fail(e); break; }
        e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) { rc = cuda_fail(e); break; }
    } while (0);
    if (rc != LBM_OK) {
        lbm_destroy(s);
        return rc;
    }
    *out = s;
    return LBM_OK;
}

// App. A steps 1-7 of the step the device scalars hold, with the divisions
// the planner selected for it, on stream `st`.
static cudaError_t launch_update(lbm_sim *s, cudaStream_t st, bool pdl = true)
{
    if (!s->d.inject_in_update && s->p.growth_mode != LBM_GROW_NONE) {
        cudaError_t e = s->kt->inject(s->d, st);
        if (e != cudaSuccess) return e;
    }
    return s->use_tma ? s->kt->tma_update(s->d, s->maps, s->tma_variant, pdl, st) : s->kt->update(s->d, st);
}

// Host-side mirror of one completed step (the kernels keep theirs on the device).
static void advance_host_step(lbm_sim *s)
{
    s->launches += (!s->d.inject_in_update && s->p.growth_mode != LBM_GROW_NONE) ? 3 : 2;
    s->cur ^= 1;
    ++s->step;
}

int lbm_step(lbm_sim *s, int64_t nsteps)
{
    if (!s || nsteps < 0) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    for (int64_t k = 0; k < nsteps; ++k) {
        const bool timed = s->timing && (s->timing_count++ % s->timing_stride) == 0 &&
                           s->ev_used + 2 <= (int64_t)s->ev.size();
        if (timed) CK(cudaEventRecord(s->ev[s->ev_used], s->stream));
        cudaError_t e = launch_update(s, s->stream);
        if (e != cudaSuccess) return cuda_fail(e);
        if (timed) {
            CK(cudaEventRecord(s->ev[s->ev_used + 1], s->stream));
            s->ev_used += 2;
        }
        // observables of the new state; divisions of the next step
        CK(s->kt->plan(s->d, 0, s->stream));
        advance_host_step(s);
    }
    return LBM_OK;
}

int lbm_sync(lbm_sim *s)
{
    if (!s) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    return LBM_OK;
}

// Eq. 6 from the exact integer sums S1 = sum h, S2 = sum h^2 of the front
// heights: hbar = S1 / W, w = sqrt(W S2 - S1^2) / W (IEEE double, the same
// operations in the same order as the kernels' FP64 wall rule).
static void eq6(long long S1, long long S2, int W, double *hbar, double *w)
{
    *hbar = (double)S1 / (double)W;
    *w = std::sqrt((double)((long long)W * S2 - S1 * S1)) / (double)W;
}

static int read_scalars(lbm_sim *s, DevScalars *hs)
{
    CK(cudaMemcpyAsync(hs, s->d.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

int lbm_stats(lbm_sim *s, lbm_stats_t *out)
{
    if (!s || !out) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    DevScalars hs;
    int rc = read_scalars(s, &hs);
    if (rc != LBM_OK) return rc;
    std::memset(out, 0, sizeof(*out));
    out->step = hs.step;
    out->ns_last = hs.ns_last;
    out->ns_total = hs.ns_total;
    out->div_total = hs.div_total;
    out->starved_steps = hs.starved_steps;
    out->cand_last = hs.cand_last;
    out->events_last = hs.events_last;
    out->mass_fix = hs.mass_fix;
    out->quiescent_fix = hs.quiescent_fix;
    out->S1 = hs.S1;
    out->S2 = hs.S2;
    out->node_updates = hs.node_updates;
    out->launches = s->launches;
    out->mass = (double)hs.mass_fix * kFixInv;
    out->quiescent_mass = (double)hs.quiescent_fix * kFixInv;
    out->carry = hs.carry;
    eq6(hs.S1, hs.S2, s->p.width, &out->hbar, &out->w);
    out->clip_mass = hs.clip_mass;
    out->y_r = hs.y_r;
    out->H_top = hs.H_top;
    out->hmin = hs.hmin;
    out->y_hi = hs.y_hi;
    out->status = hs.status;
    out->update_kernel = s->use_tma ? 2 : 1;
    return LBM_OK;
}

int lbm_clear_status(lbm_sim *s)
{
    if (!s) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    CK(cudaMemsetAsync(&s->d.sc->status, 0, sizeof(int), s->stream));
    // after a step abandoned on a timeout the planner's grid-barrier counter
    // may be off a multiple of its grid and its merge table may hold entries
    // no list points at: both restart (between steps they hold nothing the
    // next planner needs)
    CK(cudaMemsetAsync(&s->d.sc->bar_ctr, 0, sizeof(unsigned long long), s->stream));
    CK(cudaMemsetAsync(s->d.htab, 0xFF, (size_t)s->L.hcap * 8u, s->stream));
    return LBM_OK;
}

int lbm_debug_waits(lbm_sim *s, int64_t budget_cycles, int32_t withhold)
{
    if (!s || budget_cycles < 0 || withhold < 0 || withhold > 3) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    // stream-ordered, so the kernels of later steps see it (pageable host
    // values are staged by the copy call itself)
    const long long b = budget_cycles;
    const int w = withhold;
    CK(cudaMemcpyAsync(&s->d.sc->wait_budget, &b, sizeof(b), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(&s->d.sc->wait_test, &w, sizeof(w), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

int lbm_front_heights(lbm_sim *s, int32_t *h_host, double *hbar, double *w)
{
    if (!s) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    // only W int32 and the two exact Eq. 6 sums (int64) cross the bus
    long long sums[2];
    if (h_host)
        CK(cudaMemcpyAsync(h_host, s->d.heights, sizeof(int32_t) * s->p.width, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(sums, &s->d.sc->S1, 2 * sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    double hb, wv;
    eq6(sums[0], sums[1], s->p.width, &hb, &wv);
    if (hbar) *hbar = hb;
    if (w) *w = wv;
    return LBM_OK;
}

int lbm_front_heights_async(lbm_sim *s, int32_t *h_host, int64_t *sums_host)
{
    if (!s || !sums_host) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    const int W = s->p.width;
    int32_t *h_dev = h_host ? (int32_t *)device_alias(h_host) : nullptr;
    long long *s_dev = (long long *)device_alias(sums_host);
    if (s_dev && (h_dev || !h_host)) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)std::min((W + 255) / 256, 32));
        cfg.blockDim = dim3(256);
        cfg.stream = s->stream;
        cudaLaunchAttribute la[1];
        la[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        la[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = la;
        cfg.numAttrs = 1;
        CK(cudaLaunchKernelEx(&cfg, k_export_front, (const int32_t *)s->d.heights, (const long long *)&s->d.sc->S1, W,
                              h_dev, s_dev));
        return LBM_OK;
    }
    if (h_host)
        CK(cudaMemcpyAsync(h_host, s->d.heights, sizeof(int32_t) * W, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(sums_host, &s->d.sc->S1, 2 * sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    return LBM_OK;
}

int lbm_eq6(int64_t s1, int64_t s2, int32_t width, double *hbar, double *w)
{
    if (width < 1 || !hbar || !w) return LBM_ERR_INVALID_ARG;
    eq6((long long)s1, (long long)s2, width, hbar, w);
    return LBM_OK;
}

int lbm_eq6_n(const int64_t *sums, int64_t n, int32_t width, double *hbar, double *w)
{
    if (width < 1 || n < 0 || (n > 0 && (!sums || !hbar || !w))) return LBM_ERR_INVALID_ARG;
    for (int64_t i = 0; i < n; ++i) eq6((long long)sums[2 * i], (long long)sums[2 * i + 1], width, &hbar[i], &w[i]);
    return LBM_OK;
}

int lbm_fields_device(lbm_sim *s, double *rho, double *ux, double *uy)
{
    if (!s || !rho || !ux || !uy) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    CK(s->kt->fields(s->d, s->cur, rho, ux, uy, s->stream));
    return LBM_OK;
}

int lbm_fields(lbm_sim *s, double *rho, double *ux, double *uy)
{
    if (!s || !rho || !ux || !uy) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    const size_t n = (size_t)s->p.width * s->p.height;
    double *dbuf = nullptr;
    CK(cudaMallocAsync((void **)&dbuf, 3 * n * sizeof(double), s->stream));
    int rc = LBM_OK;
    cudaError_t e = s->kt->fields(s->d, s->cur, dbuf, dbuf + n, dbuf + 2 * n, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rho, dbuf, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ux, dbuf + n, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(uy, dbuf + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) rc = cuda_fail(e);
    cudaFreeAsync(dbuf, s->stream);
    e = cudaStreamSynchronize(s->stream);
    if (rc == LBM_OK && e != cudaSuccess) rc = cuda_fail(e);
    return rc;
}

int lbm_populations(lbm_sim *s, double *f_host)
{
    if (!s || !f_host) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    const int W = s->p.width, H = s->p.height, el = s->L.elem;
    const int Q = s->L.Q;
    std::vector<char> tmp((size_t)Q * W * H * el);
    for (int i = 0; i < Q; ++i) {
        const char *src = (const char *)s->d.f[s->cur] + (size_t)i * s->L.P * el;
        CK(cudaMemcpy2DAsync(tmp.data() + (size_t)i * W * H * el, (size_t)W * el, src, (size_t)s->L.Wp * el,
                             (size_t)W * el, H, cudaMemcpyDeviceToHost, s->stream));
    }
    CK(cudaStreamSynchronize(s->stream));
    const size_t n = (size_t)s->L.Q * W * H;
    if (el == 8) {
        std::memcpy(f_host, tmp.data(), n * 8);
    } else if (el == 4) {
        const float *t = (const float *)tmp.data();
        for (size_t k = 0; k < n; ++k) f_host[k] = (double)t[k];
    } else {
        const uint16_t *t = (const uint16_t *)tmp.data();
        const size_t plane = (size_t)W * H;
        for (size_t k = 0; k < n; ++k)
            f_host[k] = decode16(s->p.precision, t[k], s->d.pop_shift[plane_class((int)(k / plane))]);
    }
    return LBM_OK;
}

int lbm_set_populations(lbm_sim *s, const double *f_host)
{
    if (!s || !f_host) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    const int W = s->p.width, H = s->p.height, el = s->L.elem;
    const size_t n = (size_t)s->L.Q * W * H;
    // every step leaves the populations non-negative; so must the caller
    for (size_t k = 0; k < n; ++k)
        if (!(f_host[k] >= 0.0) || !std::isfinite(f_host[k])) return LBM_ERR_INVALID_ARG;
    std::vector<char> tmp(n * el);
    if (el == 8) {
        std::memcpy(tmp.data(), f_host, n * 8);
    } else if (el == 4) {
        float *t = (float *)tmp.data();
        for (size_t k = 0; k < n; ++k) t[k] = (float)f_host[k];
    } else {
        uint16_t *t = (uint16_t *)tmp.data();
        const size_t plane = (size_t)W * H;
        for (size_t k = 0; k < n; ++k)
            t[k] = encode16(s->p.precision, f_host[k], s->d.pop_shift[plane_class((int)(k / plane))]);
    }
    for (int b = 0; b < 2; ++b)
        for (int i = 0; i < s->L.Q; ++i) {
            char *dst = (char *)s->d.f[b] + (size_t)i * s->L.P * el;
            CK(cudaMemcpy2DAsync(dst, (size_t)s->L.Wp * el, tmp.data() + (size_t)i * W * H * el, (size_t)W * el,
                                 (size_t)W * el, H, cudaMemcpyHostToDevice, s->stream));
        }
    CK(s->kt->ghosts(s->d, s->stream));
    // the stored mass accumulators restart from this state
    DevScalars *sc = s->d.sc;
    const unsigned long long zero = 0ull;
    const int minus1 = -1, zeroi = 0;
    CK(cudaMemcpyAsync(&sc->mass_accum, &zero, sizeof(zero), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(&sc->maxmass_accum, &minus1, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(&sc->status, &zeroi, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    CK(s->kt->scan(s->d, s->cur, s->stream));
    // observe this state again and redo the selection of the next step
    CK(s->kt->plan(s->d, 1, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

int lbm_mask(lbm_sim *s, uint8_t *mask_host)
{
    if (!s || !mask_host) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    const int W = s->p.width, H = s->p.height, MW = s->L.MW;
    std::vector<uint32_t> words((size_t)H * MW);
    CK(cudaMemcpyAsync(words.data(), s->d.mask, words.size() * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) mask_host[(size_t)y * W + x] = (words[(size_t)y * MW + (x >> 5)] >> (x & 31)) & 1u;
    return LBM_OK;
}

int lbm_last_events(lbm_sim *s, int64_t *node, int32_t *pair, int32_t *count, int64_t cap, int64_t *n)
{
    if (!s || !n || cap < 0) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    DevScalars hs;
    int rc = read_scalars(s, &hs);
    if (rc != LBM_OK) return rc;
    const int ne = s->p.growth_mode == LBM_GROW_NONE || s->step == 0 ? 0 : hs.n_events;
    *n = 0;
    if (ne == 0) return LBM_OK;
    if (cap > 0 && (!node || !pair || !count)) return LBM_ERR_INVALID_ARG;
    std::vector<uint32_t> vk(ne);
    std::vector<int32_t> vc(ne);
    // the list of the latest step (lists alternate by step parity), one entry
    // per draw rank; repeats of an earlier rank's (node, pair) carry count 0
    const size_t off = (size_t)((s->step - 1) & 1) * (size_t)s->L.ns_max;
    CK(cudaMemcpyAsync(vk.data(), s->d.ev_key + off, ne * sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(vc.data(), s->d.ev_count + off, ne * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    std::vector<long long> vn(ne);
    std::vector<int32_t> vp(ne);
    std::vector<int> ord;
    for (int i = 0; i < ne; ++i) {
        vn[i] = (long long)key_y(vk[i]) * s->p.width + key_x(vk[i]);
        vp[i] = key_pair(vk[i]);
        if (vc[i] > 0) ord.push_back(i);
    }
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return vn[a] * 4 + vp[a] < vn[b] * 4 + vp[b]; });
    *n = (int64_t)ord.size();
    const int64_t m = std::min<int64_t>(cap, (int64_t)ord.size());
    for (int64_t i = 0; i < m; ++i) {
        node[i] = vn[ord[i]];
        pair[i] = vp[ord[i]];
        count[i] = vc[ord[i]];
    }
    return LBM_OK;
}

int lbm_timing_enable(lbm_sim *s, int64_t max_launches)
{
    if (!s || max_launches < 0) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    while ((int64_t)s->ev.size() < 2 * max_launches) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        s->ev.push_back(e);
    }
    s->ev_used = 0;
    s->timing_count = 0;
    s->timing = max_launches > 0;
    DevScalars hs;
    int rc = read_scalars(s, &hs);
    if (rc != LBM_OK) return rc;
    s->timing_nodes0 = hs.node_updates;
    return LBM_OK;
}

int lbm_timing_stride(lbm_sim *s, int64_t stride)
{
    if (!s || stride < 1) return LBM_ERR_INVALID_ARG;
    s->timing_stride = stride;
    return LBM_OK;
}

int lbm_timing_read(lbm_sim *s, int64_t *launches, double *total_ms, int64_t *nodes)
{
    if (!s) return LBM_ERR_INVALID_ARG;
    USE_DEVICE(s);
    DevScalars hs;
    int rc = read_scalars(s, &hs);
    if (rc != LBM_OK) return rc;
    double tot = 0.0;
    for (int64_t k = 0; k + 1 < s->ev_used; k += 2) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, s->ev[k], s->ev[k + 1]));
        tot += ms;
    }
    if (launches) *launches = s->ev_used / 2;
    if (total_ms) *total_ms = tot;
    if (nodes) *nodes = hs.node_updates - s->timing_nodes0;
    s->timing = false;
    return LBM_OK;
}

int lbm_bytes_per_node(lbm_sim *s, int64_t *bytes)
{
    if (!s || !bytes) return LBM_ERR_INVALID_ARG;
    *bytes = 2 * (int64_t)s->L.Q * (int64_t)s->L.elem;
    return LBM_OK;
}

const char *lbm_strerror(int code)
{
    switch (code) {
    case LBM_OK: return "ok";
    case LBM_ERR_INVALID_ARG: return "invalid argument";
    case LBM_ERR_OOM: return "out of device memory (or arena too small)";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_CAPACITY: return "too many divisions in one step for the planner";
    case LBM_ERR_NO_DEVICE: return "no usable CUDA device (compute capability 10.3 required)";
    case LBM_ERR_BATCH_FULL: return "every slot of the batch is taken";
    default: return "unknown error";
    }
}

const char *lbm_last_cuda_error(void) { return g_cuda_err; }

const char *lbm_version(void) { return "0.1.0 sm_103a"; }

} // extern "C"

// ---------------------------------------------------------------------------
// Batched stepping: independent simulations advanced together by replaying a
// CUDA graph (the kernels read the step index from each simulation's device
// scalars, so the same graph serves every step). When every member stores its
// populations in the same type, a step is three or four launches for the
// whole batch (injection over all slots' divisions; the update, staged over
// all members' tiles or over a table of the members' blocks; the planners,
// over tables of one block per member and of the members planned by more);
// otherwise the graph holds one chain of steps per member as parallel
// branches.
//
// The batched form keeps its members in slots: the tables in device memory
// have room for more entries than the members use (unused entries do nothing),
// so a member that joins or leaves changes table entries, not the graphs. The
// graphs are captured again only when a table outgrows its room or when a
// joining member cannot take the staged update or its bulk stores. (Both
// forms of the update, with and without Eq. 4's noise, are captured; a step
// replays the one that the current members need.)
struct lbm_batch {
    std::vector<lbm_sim *> sims; // per slot (nullptr: empty)
    int members;
    int device;
    const KernelTable *kt; // the members' kernels (the batched form)
    cudaStream_t user;     // the caller's stream
    cudaStream_t origin;   // the batch's own stream, which the graphs are captured from and run on
    std::vector<cudaStream_t> branch;
    cudaEvent_t fork;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec[2][2]; // [without, with noise][one step, kBatchChain steps]
    int captures;            // times the graphs were captured
    // batched launches: the slots' SimDev and the plain-load update's block
    // table (its room: that launch's grid), in one allocation; the planners
    // deal their blocks on the device (a cooperative launch of plan_cap
    // blocks)
    bool fused;
    void *dev_mem;
    SimDev *ds;
    int4 *bm_upd;
    int nb_upd, plan_cap;
    // the TMA-staged batched update (all members D2Q9, FP32 or 16-bit, walls
    // in y, at most kTmaBatchMaxSims slots): four maps and a MemberConst per slot
    bool tma;
    MemberConst *mc;
    CUtensorMap *maps;
    int noise, tstore, tma_grid;
    int nsm;
    // host copies of the tables
    std::vector<SimDev> h_ds;
    std::vector<int4> h_upd;
    std::vector<CUtensorMap> h_maps;
    std::vector<MemberConst> h_mc;
};

namespace {
constexpr int kBatchChain = 4; // steps per branch in the longer graph

// Captures `steps` steps of every simulation into an executable graph:
// batched launches (the update with Eq. 4's noise if `noise`), or one branch
// per simulation.
cudaError_t batch_capture(lbm_batch *b, int steps, int noise, cudaGraphExec_t *out)
{
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t first = cudaSuccess;
    if (b->fused) {
        const KernelTable *kt = b->kt;
        for (int k = 0; k < steps && first == cudaSuccess; ++k) {
            first = kt->batch_inject(b->ds, (int)b->sims.size(), 2 * b->nsm, b->origin);
            if (first == cudaSuccess)
                first = b->tma ? kt->batch_update_tma(b->ds, b->mc, b->maps, (int)b->sims.size(), noise,
                                                      b->tstore, b->tma_grid, b->origin)
                               : kt->batch_update(b->ds, b->bm_upd, b->nb_upd, b->origin);
            if (first == cudaSuccess) first = kt->batch_plan(b->ds, (int)b->sims.size(), b->plan_cap, b->origin);
        }
    } else {
        first = cudaEventRecord(b->fork, b->origin);
    }
    for (size_t i = 0; i < b->sims.size() && first == cudaSuccess && !b->fused; ++i) {
        lbm_sim *s = b->sims[i];
        first = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
        for (int k = 0; k < steps && first == cudaSuccess; ++k) {
            first = launch_update(s, b->branch[i], false);
            if (first == cudaSuccess) first = s->kt->plan(s->d, 0, b->branch[i]);
        }
        if (first == cudaSuccess) first = cudaEventRecord(b->join[i], b->branch[i]);
        if (first == cudaSuccess) first = cudaStreamWaitEvent(b->origin, b->join[i], 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->origin, &g);
    if (first == cudaSuccess) first = e;
    if (first == cudaSuccess) first = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return first;
}

cudaError_t batch_recapture(lbm_batch *b)
{
    for (auto &pair : b->exec)
        for (cudaGraphExec_t &g : pair)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    // (the branch form and the plain-load update draw the noise per member)
    const int forms = b->fused && b->tma ? 2 : 1;
    cudaError_t e = cudaSuccess;
    for (int nz = 0; nz < forms && e == cudaSuccess; ++nz) {
        e = batch_capture(b, 1, nz, &b->exec[nz][0]);
        if (e == cudaSuccess) e = batch_capture(b, kBatchChain, nz, &b->exec[nz][1]);
    }
    ++b->captures;
    return e;
}

// Whether some member draws Eq. 4's noise.
void batch_noise(lbm_batch *b)
{
    b->noise = 0;
    for (const lbm_sim *s : b->sims)
        if (s && s->d.noise_on) b->noise = 1;
}

// Whether member s can take the staged update, and its bulk stores.
bool staged_ok(const lbm_sim *s) { return s->p.lattice == LBM_D2Q9 && !s->p.y_periodic; }
bool bulk_store_ok(const lbm_sim *s)
{
    // from the tuned table's width on (the narrowest width from which the
    // single-lattice sweep's fastest FP32 form stores in bulk); measured:
    // four 4096 x 2048 members 66.3 against 63.8 G node updates/s with bulk
    // stores, but the 256-member ensemble of widths 256..2048 53.0 against
    // 56.7 (four CTAs per SM instead of five)
    return s->p.precision == LBM_FP32 && s->p.width % 4 == 0 && s->p.width >= kTunedBatchBulkMinWidth;
}

// The plain-load update's table for the current members (unpadded): about
// two waves of its kernel for the whole batch, dealt by lattice area, each
// member a multiple of its column tiles. `upd_bound`: the most entries any
// subset of the members can need (a member's entries exceed its share of
// the two waves by less than its column tiles).
void batch_entries(const lbm_batch *b, std::vector<int4> &upd, long long *upd_bound)
{
    const KernelTable *kt = b->kt;
    const int bps = std::max(1, kt->update_blocks_per_sm());
    double area = 0.0;
    for (const lbm_sim *s : b->sims)
        if (s) area += (double)s->p.width * (double)s->p.height;
    const double target = 2.0 * b->nsm * bps;
    upd.clear();
    *upd_bound = (long long)target;
    for (size_t i = 0; i < b->sims.size(); ++i) {
        const lbm_sim *s = b->sims[i];
        if (!s) continue;
        const int ncx = (s->p.width + kt->update_tile_x - 1) / kt->update_tile_x;
        *upd_bound += ncx;
        const double share = target * (double)s->p.width * (double)s->p.height / area;
        const int nbu = std::max(1, (int)std::lround(share / ncx)) * ncx;
        for (int j = 0; j < nbu; ++j) upd.push_back(make_int4((int)i, j, nbu, 0));
    }
}

// Slot i's SimDev, MemberConst and tensor maps (zeros for an empty slot).
cudaError_t batch_slot(lbm_batch *b, size_t i)
{
    const lbm_sim *s = b->sims[i];
    std::memset(&b->h_ds[i], 0, sizeof(SimDev));
    if (s) b->h_ds[i] = s->d;
    if (!b->tma) return cudaSuccess;
    MemberConst &c = b->h_mc[i];
    std::memset(&c, 0, sizeof(c));
    std::memset(&b->h_maps[4 * i], 0, 4 * sizeof(CUtensorMap));
    if (!s) return cudaSuccess;
    c.f[0] = s->d.f[0];
    c.f[1] = s->d.f[1];
    c.mask = s->d.mask;
    c.sc = s->d.sc;
    c.P = s->d.P;
    c.W = s->d.W;
    c.H = s->d.H;
    c.Wp = s->d.Wp;
    c.MW = s->d.MW;
    c.key0 = s->d.key0;
    c.key1 = s->d.key1;
    c.sim = s->d.sim;
    c.negfix = s->d.negfix;
    c.rho_c = s->d.f_rho_c;
    c.om1 = s->d.f_om1;
    c.ow1 = s->d.f_ow1;
    c.ow5 = s->d.f_ow5;
    c.cmu = s->d.f_cmu;
    c.two_sigma = s->d.f_two_sigma;
    for (int k = 0; k < 3; ++k) c.pop_shift[k] = s->d.pop_shift[k];
    for (int h = 0; h < 2; ++h) {
        char *base_c = (char *)s->d.f[h] - (size_t)kXO * s->L.elem;
        if (!encode_population_map(&b->h_maps[4 * i + h], base_c, s->d.Wp, s->d.Wp, s->d.H, s->d.P, s->L.Q,
                                   kTmaBoxX + 8, 4, s->p.precision))
            return cudaErrorInvalidValue;
        // bulk stores of a tile's 128 columns, cut at x = W - 1
        if (b->tstore && !encode_population_map(&b->h_maps[4 * i + 2 + h], base_c, s->p.width + kXO, s->d.Wp,
                                                s->d.H, s->d.P, s->L.Q, kTmaBoxX, 2, s->p.precision))
            return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

// Brings the device tables up to date with the slots: recomputes the entries,
// lays the tables out again (and captures the graphs again) if one outgrows
// its room or the planner launch must become cooperative, pads each table
// with unused entries and copies everything over, stream-ordered on the
// batch's stream after the steps already enqueued.
cudaError_t batch_refresh(lbm_batch *b, bool relayout)
{
    std::vector<int4> upd;
    long long upd_bound = 0;
    batch_entries(b, upd, &upd_bound);
    if (b->tma) upd.clear(); // (the staged update deals the tiles itself)
    if (!relayout) relayout = (int)upd.size() > b->nb_upd;
    cudaError_t e = cudaSuccess;
    if (relayout) {
        // room: enough for any subset of the members (members that leave
        // never force a new layout), twice what they use when growing a
        // layout that had some (a batch that gains members regrows rarely)
        const bool grow = b->dev_mem != nullptr;
        auto room = [&](long long need, int old) {
            return (int)std::max<long long>(std::max<long long>(1, old), grow ? 2 * need : need);
        };
        b->nb_upd = b->tma ? std::max(1, b->nb_upd) : room(std::max<long long>(upd_bound, (long long)upd.size()),
                                                           b->nb_upd);
        const size_t n = b->sims.size();
        const size_t off_u = align256(n * sizeof(SimDev));
        const size_t off_m = align256(off_u + (size_t)b->nb_upd * sizeof(int4)); // tensor maps (128-byte aligned)
        const size_t off_c = align256(off_m + (b->tma ? 4 * n : 0) * sizeof(CUtensorMap)); // member constants
        const size_t bytes = off_c + (b->tma ? n : 0) * sizeof(MemberConst);
        if (b->dev_mem) {
            e = cudaFreeAsync(b->dev_mem, b->origin);
            b->dev_mem = nullptr;
            if (e != cudaSuccess) return e;
        }
        e = cudaMallocAsync(&b->dev_mem, bytes, b->origin);
        if (e != cudaSuccess) return e;
        char *base = (char *)b->dev_mem;
        b->ds = (SimDev *)base;
        b->bm_upd = (int4 *)(base + off_u);
        b->maps = b->tma ? (CUtensorMap *)(base + off_m) : nullptr;
        b->mc = b->tma ? (MemberConst *)(base + off_c) : nullptr;
        b->h_maps.assign(b->tma ? 4 * n : 0, CUtensorMap{});
        b->h_mc.assign(b->tma ? n : 0, MemberConst{});
        b->h_ds.assign(n, SimDev{});
        for (size_t i = 0; i < n && e == cudaSuccess; ++i) e = batch_slot(b, i);
        if (e != cudaSuccess) return e;
    }
    const int4 unused = make_int4(-1, 0, 1, 0);
    upd.resize((size_t)b->nb_upd, unused);
    b->h_upd.swap(upd);
    const size_t n = b->sims.size();
    e = cudaMemcpyAsync(b->ds, b->h_ds.data(), n * sizeof(SimDev), cudaMemcpyHostToDevice, b->origin);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->bm_upd, b->h_upd.data(), b->h_upd.size() * sizeof(int4), cudaMemcpyHostToDevice,
                            b->origin);
    if (e == cudaSuccess && b->tma)
        e = cudaMemcpyAsync(b->maps, b->h_maps.data(), b->h_maps.size() * sizeof(CUtensorMap),
                            cudaMemcpyHostToDevice, b->origin);
    if (e == cudaSuccess && b->tma)
        e = cudaMemcpyAsync(b->mc, b->h_mc.data(), b->h_mc.size() * sizeof(MemberConst), cudaMemcpyHostToDevice,
                            b->origin);
    // the host copies change with the next member: wait for the copies from them
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->origin);
    b->tma_grid = (b->tstore ? kTmaBatchCtasPerSmStore : kTmaBatchCtasPerSm) * b->nsm;
    if (e == cudaSuccess && relayout) e = batch_recapture(b);
    return e;
}

lbm_batch *batch_new(int slots, int device, cudaStream_t user)
{
    lbm_batch *b = new lbm_batch();
    b->sims.assign((size_t)slots, nullptr);
    b->members = 0;
    b->device = device;
    b->kt = nullptr;
    b->user = user;
    b->origin = nullptr;
    b->exec[0][0] = b->exec[0][1] = b->exec[1][0] = b->exec[1][1] = nullptr;
    b->captures = 0;
    b->fork = nullptr;
    b->fused = true;
    b->dev_mem = nullptr;
    b->ds = nullptr;
    b->bm_upd = nullptr;
    b->nb_upd = b->plan_cap = 0;
    b->tma = false;
    b->mc = nullptr;
    b->maps = nullptr;
    b->noise = b->tstore = b->tma_grid = 0;
    b->nsm = 0;
    return b;
}

// The streams, events and first tables and graphs of a new batch.
cudaError_t batch_init(lbm_batch *b)
{
    cudaError_t e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    // one-time kernel attributes are set outside the capture
    for (lbm_sim *s : b->sims)
        if (e == cudaSuccess && s && s->use_tma) e = s->kt->tma_prepare(s->d, s->tma_variant);
    // branch streams and join events for the branch form; the batched form
    // needs one event (a stream wait takes the event's record at the call)
    const size_t nj = b->fused ? 1 : b->sims.size();
    for (size_t i = 0; i < nj && e == cudaSuccess; ++i) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->join.push_back(ev);
        if (b->fused || e != cudaSuccess) continue;
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->branch.push_back(st);
    }
    if (e != cudaSuccess) return e;
    if (!b->fused) return batch_recapture(b);
    // the cooperative planner launch: every resident block
    b->plan_cap = std::max(2, b->kt->plan_blocks_per_sm(1) * b->nsm);
    if (b->members == 0) {
        // an empty batch: room for members to come (the plain-load update's
        // two waves and 32 column tiles more per slot)
        const int bps = std::max(1, b->kt->update_blocks_per_sm());
        b->nb_upd = 2 * bps * b->nsm + 32 * (int)b->sims.size();
    }
    return batch_refresh(b, true);
}
} // namespace

extern "C" {

int lbm_batch_create(lbm_sim *const *sims, int32_t n, void *stream, lbm_batch **out)
{
    if (!sims || n < 1 || !out) return LBM_ERR_INVALID_ARG;
    for (int32_t i = 0; i < n; ++i) {
        if (!sims[i] || sims[i]->device != sims[0]->device || sims[i]->timing) return LBM_ERR_INVALID_ARG;
        for (int32_t j = 0; j < i; ++j)
            if (sims[j] == sims[i]) return LBM_ERR_INVALID_ARG;
    }
    CK(cudaSetDevice(sims[0]->device));
    lbm_batch *b = batch_new(n, sims[0]->device, (cudaStream_t)stream);
    for (int32_t i = 0; i < n; ++i) b->sims[i] = sims[i];
    b->members = n;
    b->kt = sims[0]->kt;
    // one launch per kernel for the whole batch when the members share the
    // storage type (the plain-load or the TMA-staged update: the same results,
    // bit for bit), the TMA-staged one when every member can take it
    for (int32_t i = 1; i < n; ++i)
        if (sims[i]->kt != sims[0]->kt) b->fused = false;
    b->tma = b->fused && b->kt->batch_update_tma && n <= kTmaBatchMaxSims;
    b->tstore = b->tma ? 1 : 0;
    for (int32_t i = 0; i < n; ++i) {
        if (!staged_ok(sims[i])) b->tma = false;
        if (!bulk_store_ok(sims[i])) b->tstore = 0;
    }
    batch_noise(b);
    if (!b->tma) b->tstore = 0;
    const cudaError_t e = batch_init(b);
    if (e != cudaSuccess) {
        lbm_batch_destroy(b);
        return cuda_fail(e);
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_create_empty(int32_t slots, int32_t lattice, int32_t precision, void *stream, lbm_batch **out)
{
    if (!out || slots < 1 || slots > kMaxBatchSlots) return LBM_ERR_INVALID_ARG;
    if ((lattice != LBM_D2Q9 && lattice != LBM_D2Q7) || precision < LBM_FP32 || precision > LBM_BF16)
        return LBM_ERR_INVALID_ARG;
    if (lattice == LBM_D2Q7 && precision != LBM_FP32 && precision != LBM_FP64) return LBM_ERR_INVALID_ARG;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    lbm_batch *b = batch_new(slots, dev, (cudaStream_t)stream);
    b->kt = kernel_table(lattice, precision);
    b->tma = b->kt->batch_update_tma && slots <= kTmaBatchMaxSims;
    const cudaError_t e = batch_init(b);
    if (e != cudaSuccess) {
        lbm_batch_destroy(b);
        return cuda_fail(e);
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_attach(lbm_batch *b, lbm_sim *s, int32_t *slot)
{
    if (!b || !s || !b->fused || s->kt != b->kt || s->device != b->device || s->timing) return LBM_ERR_INVALID_ARG;
    int free_slot = -1;
    for (size_t i = 0; i < b->sims.size(); ++i) {
        if (b->sims[i] == s) return LBM_ERR_INVALID_ARG;
        if (!b->sims[i] && free_slot < 0) free_slot = (int)i;
    }
    if (free_slot < 0) return LBM_ERR_BATCH_FULL;
    CK(cudaSetDevice(b->device));
    // a member that the current graphs cannot step: capture them again
    bool relayout = false;
    if (b->tma && !staged_ok(s)) {
        b->tma = false;
        b->tstore = 0;
        relayout = true;
    }
    if (b->tstore && !bulk_store_ok(s)) {
        b->tstore = 0;
        relayout = true;
    }
    if (s->use_tma) CK(s->kt->tma_prepare(s->d, s->tma_variant));
    // the batch's steps come after what the member's stream holds
    CK(cudaEventRecord(b->join[0], s->stream));
    CK(cudaStreamWaitEvent(b->origin, b->join[0], 0));
    b->sims[(size_t)free_slot] = s;
    ++b->members;
    cudaError_t e = relayout ? cudaSuccess : batch_slot(b, (size_t)free_slot);
    if (e == cudaSuccess) e = batch_refresh(b, relayout);
    if (e != cudaSuccess) {
        b->sims[(size_t)free_slot] = nullptr;
        --b->members;
        return cuda_fail(e);
    }
    batch_noise(b);
    if (slot) *slot = free_slot;
    return LBM_OK;
}

int lbm_batch_detach(lbm_batch *b, lbm_sim *s)
{
    if (!b || !s || !b->fused) return LBM_ERR_INVALID_ARG;
    size_t i = 0;
    while (i < b->sims.size() && b->sims[i] != s) ++i;
    if (i == b->sims.size()) return LBM_ERR_INVALID_ARG;
    CK(cudaSetDevice(b->device));
    b->sims[i] = nullptr;
    --b->members;
    batch_noise(b);
    cudaError_t e = batch_slot(b, i);
    if (e == cudaSuccess) e = batch_refresh(b, false);
    // what the member's stream gets next comes after the batch's steps
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->origin);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, b->fork, 0);
    return e == cudaSuccess ? LBM_OK : cuda_fail(e);
}

int lbm_batch_members(const lbm_batch *b)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    return b->members;
}

int lbm_batch_captures(const lbm_batch *b)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    return b->captures;
}

int lbm_batch_step(lbm_batch *b, int64_t nsteps)
{
    if (!b || nsteps < 0) return LBM_ERR_INVALID_ARG;
    if (b->members == 0 || nsteps == 0) return LBM_OK;
    CK(cudaSetDevice(b->device));
    // after whatever the caller's stream and each member's own stream hold ...
    CK(cudaEventRecord(b->fork, b->user));
    CK(cudaStreamWaitEvent(b->origin, b->fork, 0));
    for (size_t i = 0; i < b->sims.size(); ++i) {
        if (!b->sims[i]) continue;
        cudaEvent_t ev = b->join[b->fused ? 0 : i];
        CK(cudaEventRecord(ev, b->sims[i]->stream));
        CK(cudaStreamWaitEvent(b->origin, ev, 0));
    }
    cudaGraphExec_t *exec = b->exec[b->exec[1][0] ? b->noise : 0];
    int64_t left = nsteps;
    for (; left >= kBatchChain; left -= kBatchChain) CK(cudaGraphLaunch(exec[1], b->origin));
    for (; left > 0; --left) CK(cudaGraphLaunch(exec[0], b->origin));
    // ... and before whatever comes next on it
    CK(cudaEventRecord(b->fork, b->origin));
    CK(cudaStreamWaitEvent(b->user, b->fork, 0));
    for (lbm_sim *s : b->sims) {
        if (!s) continue;
        CK(cudaStreamWaitEvent(s->stream, b->fork, 0));
        for (int64_t k = 0; k < nsteps; ++k) advance_host_step(s);
    }
    return LBM_OK;
}

int lbm_batch_fused(const lbm_batch *b)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    return b->fused ? (b->tma ? (b->tstore ? 3 : 2) : 1) : 0;
}

int lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return LBM_OK;
    cudaSetDevice(b->device);
    if (b->origin) cudaStreamSynchronize(b->origin);
    for (auto &pair : b->exec)
        for (cudaGraphExec_t g : pair)
            if (g) cudaGraphExecDestroy(g);
    for (cudaStream_t st : b->branch) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->dev_mem) cudaFreeAsync(b->dev_mem, b->origin);
    if (b->origin) {
        cudaStreamSynchronize(b->origin);
        cudaStreamDestroy(b->origin);
    }
    delete b;
    return LBM_OK;
}

} // extern "C"
