// Many images of different sizes in one persistent launch.
//
// The plan cuts every image into warp work items -- (image, column segment, row band) tiles,
// the same items the single-image kernels use -- with a band height chosen per shape bucket and
// a schedule (claim order, edge-segment weight, segment origin, staging of interior segments)
// chosen for the whole plan, from a tuning cache written by paper_2201_03611_b300/tune.py, else
// built-in defaults. A persistent grid (one resident set of CTAs per SM) claims the tiles warp
// by warp from an atomic counter in the workspace. Each tile writes its own
// parameter-cotangent partials at its fixed index, and a separate kernel sums them in a fixed
// order (per image for d kappa_i, over all tiles for d Wx, d Wy), so results do not depend on
// which warp ran which tile. There are no inter-CTA waits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "harris_bwd_strip.cuh"
#include "harris_fwd_strip.cuh"
#include "shine.h"
#include "shine_host.h"
#include "entry.h"

struct shine_plan {
    int n = 0;
    int dt = 0;
    int border = 0;
    int mode = 0;
    int ntiles = 0;
    int grid = 0;
    std::vector<int64_t> H, W;
    std::vector<int> band_rows;
    std::vector<int> tile_begin;  // [n + 1], image-major tile ids
    int order = 0;                // claim order (SHINE_ORDER_*)
    int staging = 0;              // interior segments: 0 per-lane cp.async, 1 bulk copies
    int edge_w4 = 6;              // an edge-segment tile row weighs edge_w4 / 4 interior rows
    int origin = 0;               // first output column of segment 0 of every image
    void* dbuf = nullptr;         // device: tiles (int4 x ntiles) | band_rows (n) | tile_begin (n+1)
    int4* d_tiles = nullptr;
    int* d_band_rows = nullptr;
    int* d_tile_begin = nullptr;
};

namespace shine {

namespace {

constexpr int kBatchThreads = 128;
template <bool FWD_BWD> constexpr int batch_stages() { return FWD_BWD ? kBwdStages : 0; }

struct BatchArgs {
    const shine_image_desc* descs;
    const int4* tiles;       // (image, seg, band, tile id) in claim order
    const int* band_rows;    // per image
    int ntiles;
    int n;
    int valid;
    int origin;              // first output column of segment 0
    unsigned int* err;       // set when a bounded wait gave up (bulk staging)
    unsigned int* dbg;       // debug builds: index-check violation word
    unsigned int* counter;
    double* partials;        // [kParamSlots][ntiles]
    const float* kappa;      // [n]
    const float* wx;
    const float* wy;
};

__device__ __forceinline__ void dev_geometry(Geometry& g, int H, int W, int valid, bool full_image, int br,
                                             int x0, unsigned int* dbg) {
    g.H = H; g.W = W; g.valid = valid;
    g.dbg = dbg;
    if (valid && !full_image) {
        g.xlo = 2; g.xhi = W - 2; g.ylo = 2; g.yhi = H - 2; g.ox = 2; g.oy = 2;
    } else {
        g.xlo = 0; g.xhi = W; g.ylo = 0; g.yhi = H; g.ox = valid ? 2 : 0; g.oy = valid ? 2 : 0;
    }
    g.x0 = x0;
    g.nseg = (g.xhi - x0 + kSegOut - 1) / kSegOut;
    g.band_rows = br;
    g.nband = (g.yhi - g.ylo + br - 1) / br;
}

__device__ __forceinline__ bool dev_aligned(const void* p, int64_t pitch, size_t esize, size_t chunk) {
    return (reinterpret_cast<uintptr_t>(p) % chunk) == 0 && ((size_t)pitch * esize) % chunk == 0;
}

// BULK: interior segments of images whose image and cotangent rows are 16-byte aligned are staged
// by bulk copies (lane 0, one mbarrier per ring slot, bounded waits), the rest per lane by
// cp.async; otherwise every segment per lane.
template <typename T, bool FWD_BWD, bool BULK>
__global__ void __launch_bounds__(kBatchThreads) harris_batched_kernel(BatchArgs b) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int NS = batch_stages<FWD_BWD>();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    T* ring = reinterpret_cast<T*>(smem_raw) + warp * NS * kLanes * 12 + lane * 12;
    T* gring = reinterpret_cast<T*>(smem_raw + (size_t)kBatchThreads * NS * 12 * sizeof(T)) +
               warp * NS * kLanes * 4 + lane * 4;
    constexpr size_t chunk = sizeof(T) == 4 ? 16 : 8;
    const bool producer = lane >= 1 && lane <= 30;
    BulkState bulk;
    bulk.seq = 0;
    bulk.failed = false;
    if constexpr (BULK && FWD_BWD) {
        bulk.bars = smem_u32(smem_raw + (size_t)kBatchThreads * NS * 16 * sizeof(T)) + (uint32_t)warp * NS * 8;
        if (lane == 0)
            for (int i = 0; i < NS; ++i) mbar_init(bulk.bars + 8 * i, 1);
        mbar_init_fence();
        __syncwarp();
    }
    Params P;
    load_params(P, b.wx, b.wy, b.kappa);  // kappa replaced per tile below

    for (;;) {
        unsigned int t = 0;
        if (lane == 0) t = atomicAdd(b.counter, 1u);
        t = __shfl_sync(kFull, t, 0);
        if (t >= (unsigned)b.ntiles || bulk.failed) break;
        const int4 tile = b.tiles[t];
        const int img = tile.x, seg = tile.y, band = tile.z, tile_id = tile.w;
        const shine_image_desc d = b.descs[img];
        P.kappa = __ldg(b.kappa + img);
        const int H = (int)d.H, W = (int)d.W;
        if constexpr (!FWD_BWD) {
            FwdArgs a;
            dev_geometry(a, H, W, b.valid, false, b.band_rows[img], b.origin, b.dbg);
            a.img = d.img; a.img_pitch = d.img_pitch; a.out = d.out; a.out_pitch = d.out_pitch;
            a.kappa = b.kappa + img; a.wx = b.wx; a.wy = b.wy;
            a.aligned = dev_aligned(d.img, d.img_pitch, sizeof(T), chunk);
            a.out_vec = !b.valid && dev_aligned(d.out, d.out_pitch, sizeof(T), 4 * sizeof(T));
            a.tma = 0;
            a.err = nullptr;
            const int xb = a.x0 + seg * kSegOut, x = xb - 4 + 4 * lane;
            const int y0 = a.ylo + band * a.band_rows, y1 = min(y0 + a.band_rows, a.yhi);
            const bool edge = (xb - 4 < 0) || (xb + kSegOut + 4 > W) || a.valid;
            if (a.aligned) {
                if (edge) fwd_strip<T, T, kFwdEdgeStages, true, true>(a, P, lane, x, y0, y1);
                else fwd_strip<T, T, kFwdStages, false, true>(a, P, lane, x, y0, y1);
            } else {
                fwd_strip<T, T, kFwdStages, true, false>(a, P, lane, x, y0, y1);
            }
        } else {
            BwdArgs a;
            dev_geometry(a, H, W, b.valid, true, b.band_rows[img], b.origin, b.dbg);
            a.img = d.img; a.img_pitch = d.img_pitch;
            a.gout = d.grad_out; a.gout_pitch = d.gout_pitch;
            a.gho = b.valid ? H - 4 : H; a.gwo = b.valid ? W - 4 : W;
            a.gimg = d.grad_img; a.gimg_pitch = d.gimg_pitch;
            a.kappa = b.kappa + img; a.wx = b.wx; a.wy = b.wy;
            a.partials = nullptr;
            a.pstride = 0;
            a.poffset = 0;
            a.err = nullptr;
            a.tma = 0;
            a.aligned = dev_aligned(d.img, d.img_pitch, sizeof(T), chunk);
            a.g_aligned = !b.valid && dev_aligned(d.grad_out, d.gout_pitch, sizeof(T), 4 * sizeof(T));
            a.gimg_vec = d.grad_img != nullptr && dev_aligned(d.grad_img, d.gimg_pitch, sizeof(T), chunk);
            const bool rvec = d.out != nullptr && dev_aligned(d.out, d.out_pitch, sizeof(T), 4 * sizeof(T));
            const int xb = a.x0 + seg * kSegOut, x = xb - 4 + 4 * lane;
            const int y0 = band * a.band_rows, y1 = min(y0 + a.band_rows, H);
            const bool edge = (xb - 4 < 0) || (xb + kSegOut + 4 > W);
            float acc[kParamSlots];
#pragma unroll
            for (int i = 0; i < kParamSlots; ++i) acc[i] = 0.0f;
            T* rout = static_cast<T*>(d.out);
            bool bulk_ok = false;
            if constexpr (BULK) {
                bulk_ok = !b.valid && !edge && dev_aligned(d.img, d.img_pitch, sizeof(T), 16) &&
                          dev_aligned(d.grad_out, d.gout_pitch, sizeof(T), 16) && ((xb - 4) * 3 * (int)sizeof(T)) % 16 == 0;
            }
            if (bulk_ok) {
                if constexpr (BULK)
                    bwd_strip<T, T, NS, false, true, true, true, true>(a, P, lane, x, y0, y1, ring, gring, acc, rout,
                                                                       d.out_pitch, rvec, &bulk);
            } else if (a.aligned && a.g_aligned) {
                if (edge)
                    bwd_strip<T, T, NS, true, true, true, true>(a, P, lane, x, y0, y1, ring, gring, acc, rout,
                                                                d.out_pitch, rvec);
                else
                    bwd_strip<T, T, NS, false, true, true, true>(a, P, lane, x, y0, y1, ring, gring, acc, rout,
                                                                 d.out_pitch, rvec);
            } else {
                bwd_strip<T, T, NS, true, false, false, true>(a, P, lane, x, y0, y1, ring, gring, acc, rout,
                                                              d.out_pitch, rvec);
            }
#pragma unroll
            for (int i = 0; i < kParamSlots; ++i) {
                double v = producer ? (double)acc[i] : 0.0;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
                if (lane == 0) b.partials[(int64_t)i * b.ntiles + tile_id] = v;
            }
        }
    }
    if (bulk.failed && lane == 0) atomicOr(b.err, 1u);
}

// Fixed-order sums: block i < n -> d kappa_i over image i's tiles; block n + f -> d W slot f.
__global__ void __launch_bounds__(256) finalize_batched_kernel(const double* partials, int ntiles, int n,
                                                               const int* tile_begin, float* gkappa, float* gwx,
                                                               float* gwy) {
    __shared__ double red[256];
    const int blk = blockIdx.x;
    int f, lo, hi;
    if (blk < n) { f = 0; lo = tile_begin[blk]; hi = tile_begin[blk + 1]; }
    else { f = 1 + (blk - n); lo = 0; hi = ntiles; }
    double s = 0.0;
    for (int i = lo + (int)threadIdx.x; i < hi; i += 256) s += partials[(int64_t)f * ntiles + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        float v = (float)red[0];
        if (blk < n) { if (gkappa) gkappa[blk] = v; }
        else if (f < 10) { if (gwx) gwx[f - 1] = v; }
        else { if (gwy) gwy[f - 10] = v; }
    }
}

template <typename T, bool FWD_BWD, bool BULK>
size_t batched_smem() {
    return (size_t)kBatchThreads * batch_stages<FWD_BWD>() * (12 + (FWD_BWD ? 4 : 0)) * sizeof(T) +
           (BULK && FWD_BWD ? (size_t)(kBatchThreads / 32) * batch_stages<FWD_BWD>() * 8 : 0);
}

template <typename T, bool FWD_BWD, bool BULK>
int batched_grid() {
    auto kern = harris_batched_kernel<T, FWD_BWD, BULK>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batched_smem<T, FWD_BWD, BULK>());
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, batched_smem<T, FWD_BWD, BULK>()) !=
            cudaSuccess ||
        per_sm <= 0)
        per_sm = 1;
    return per_sm * sm_count();
}

template <typename T, bool FWD_BWD, bool BULK>
cudaError_t launch_batched_t(const BatchArgs& b, int grid, cudaStream_t s) {
    auto kern = harris_batched_kernel<T, FWD_BWD, BULK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batched_smem<T, FWD_BWD, BULK>());
    if (e != cudaSuccess) return e;
    kern<<<grid, kBatchThreads, batched_smem<T, FWD_BWD, BULK>(), s>>>(b);
    return cudaPeekAtLastError();
}

template <typename T>
int grid_for_t(int mode, int staging) {
    if (mode != SHINE_MODE_FWD_BWD) return batched_grid<T, false, false>();
    return staging ? batched_grid<T, true, true>() : batched_grid<T, true, false>();
}
int grid_for(int dt, int mode, int staging) {
    switch (dt) {
        case SHINE_F32: return grid_for_t<float>(mode, staging);
        case SHINE_BF16: return grid_for_t<__nv_bfloat16>(mode, staging);
        default: return grid_for_t<__half>(mode, staging);
    }
}

template <typename T>
cudaError_t launch_batched_dt(const BatchArgs& b, int mode, int staging, int grid, cudaStream_t s) {
    if (mode != SHINE_MODE_FWD_BWD) return launch_batched_t<T, false, false>(b, grid, s);
    return staging ? launch_batched_t<T, true, true>(b, grid, s) : launch_batched_t<T, true, false>(b, grid, s);
}
cudaError_t launch_batched(const BatchArgs& b, int dt, int mode, int staging, int grid, cudaStream_t s) {
    switch (dt) {
        case SHINE_F32: return launch_batched_dt<float>(b, mode, staging, grid, s);
        case SHINE_BF16: return launch_batched_dt<__nv_bfloat16>(b, mode, staging, grid, s);
        default: return launch_batched_dt<__half>(b, mode, staging, grid, s);
    }
}

// ---------------------------------------------------------------------------------------------
// Tuning cache: text lines, '#' comments.
//   "<gpu> <dtype> <border> <mode> <bucket> <band_rows>": the band height of the images whose
//       row count falls in shape bucket ceil(log2(rows));
//   "<gpu> <dtype> <border> <mode> plan <order> <staging> <edge_w4> <origin>": the schedule.
// Lines of other GPUs, dtypes, borders or modes are ignored; missing entries take the defaults.
// ---------------------------------------------------------------------------------------------
int bucket_of(int64_t rows) {
    int b = 0;
    while ((int64_t(1) << b) < rows) ++b;
    return b;
}

std::string gpu_key() {
    int dev = 0;
    cudaDeviceProp p;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    std::string name = p.name;
    for (char& c : name)
        if (c == ' ') c = '_';
    int rt = 0;
    cudaRuntimeGetVersion(&rt);
    return name + "/sm" + std::to_string(p.major * 10 + p.minor) + "/" + std::to_string(p.multiProcessorCount) +
           "sm/cuda" + std::to_string(rt);
}

struct TuneEntry {
    int bucket, rows;
};
struct TuneSchedule {
    int order = SHINE_ORDER_LONGEST_FIRST, staging = 0, edge_w4 = 6, origin = 0;
};

// Schedule values a plan accepts (the segment origin keeps every lane's staged chunk aligned for
// its copy: a multiple of 4 columns, and 4 mod 8 for bulk-staged 16-bit images).
bool schedule_ok(const TuneSchedule& t, int dt) {
    if (t.order < SHINE_ORDER_LONGEST_FIRST || t.order > SHINE_ORDER_LARGEST_IMAGE_FIRST) return false;
    if (t.staging != 0 && t.staging != 1) return false;
    if (t.edge_w4 < 1 || t.edge_w4 > 64) return false;
    if (t.origin > 0 || t.origin <= -kSegOut || t.origin % 4 != 0) return false;
    if (t.staging == 1 && dt != SHINE_F32 && ((t.origin % 8) + 8) % 8 != 4) return false;
    return true;
}

std::vector<TuneEntry> read_tune_cache(const char* path, int dt, int border, int mode, TuneSchedule* sched) {
    std::vector<TuneEntry> out;
    if (!path) return out;
    FILE* f = std::fopen(path, "r");
    if (!f) return out;
    const std::string key = gpu_key();
    char gk[256], what[32];
    int d, b, m, v[4];
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#') continue;
        const int got = std::sscanf(line, "%255s %d %d %d %31s %d %d %d %d", gk, &d, &b, &m, what, &v[0], &v[1], &v[2],
                                    &v[3]);
        if (got < 6 || key != gk || d != dt || b != border || m != mode) continue;
        if (std::strcmp(what, "plan") == 0) {
            if (got == 9) {
                TuneSchedule t;
                t.order = v[0]; t.staging = v[1]; t.edge_w4 = v[2]; t.origin = v[3];
                if (schedule_ok(t, dt)) *sched = t;
            }
        } else {
            char* end = nullptr;
            const long bucket = std::strtol(what, &end, 10);
            if (end != what && *end == '\0' && v[0] > 0) out.push_back({(int)bucket, v[0]});
        }
    }
    std::fclose(f);
    return out;
}

int default_band_rows(int64_t rows, int mode) {
    // long bands keep the vertical halo (4 or 8 recomputed rows per band) small; short ones
    // balance the tail of the persistent schedule
    const int64_t target = mode == SHINE_MODE_FWD_BWD ? 256 : 128;
    return (int)std::max<int64_t>(1, std::min<int64_t>(rows, target));
}

}  // namespace

}  // namespace shine

using namespace shine;

extern "C" {

shine_status shine_plan_create(const int64_t* HW, int32_t n, shine_dtype dt, shine_border border, int32_t mode,
                               const char* tune_cache_path, shine_plan** plan) {
    SHINE_ENTRY("shine_plan_create");
    if (!HW || n <= 0 || !plan || !dtype_ok(dt) || !border_ok(border)) return SHINE_ERR_INVALID_ARG;
    if (mode != SHINE_MODE_FWD && mode != SHINE_MODE_FWD_BWD) return SHINE_ERR_INVALID_ARG;
    *plan = nullptr;
    shine_plan* p = new (std::nothrow) shine_plan();
    if (!p) return SHINE_ERR_INVALID_ARG;
    p->n = n; p->dt = dt; p->border = border; p->mode = mode;
    TuneSchedule sched;
    const std::vector<TuneEntry> tuned = read_tune_cache(tune_cache_path, dt, border, mode, &sched);
    p->order = sched.order;
    p->staging = mode == SHINE_MODE_FWD_BWD ? sched.staging : 0;
    p->edge_w4 = sched.edge_w4;
    p->origin = sched.origin;
    struct Item { int img, seg, band, id; int64_t work; };
    std::vector<Item> items;
    std::vector<int64_t> img_work(n, 0);
    p->tile_begin.push_back(0);
    for (int i = 0; i < n; ++i) {
        const int64_t H = HW[2 * i], W = HW[2 * i + 1];
        if (check_shape(H, W, border) != SHINE_OK) { delete p; return SHINE_ERR_INVALID_ARG; }
        p->H.push_back(H);
        p->W.push_back(W);
        Geometry g;
        fill_geometry(g, H, W, border, mode == SHINE_MODE_FWD_BWD, 1);
        const int64_t rows = g.yhi - g.ylo;
        int br = default_band_rows(rows, mode);
        const int bk = bucket_of(rows);
        for (const TuneEntry& e : tuned)
            if (e.bucket == bk) br = (int)std::max<int64_t>(1, std::min<int64_t>(rows, e.rows));
        p->band_rows.push_back(br);
        fill_geometry(g, H, W, border, mode == SHINE_MODE_FWD_BWD, br);
        g.x0 = p->origin;
        g.nseg = (g.xhi - g.x0 + kSegOut - 1) / kSegOut;
        const int halo = mode == SHINE_MODE_FWD_BWD ? 8 : 4;
        for (int band = 0; band < g.nband; ++band) {
            const int y0 = g.ylo + band * br, y1 = std::min(y0 + br, g.yhi);
            for (int seg = 0; seg < g.nseg; ++seg) {
                const int id = (int)items.size();
                // edge segments (clamps, element-wise staging) run slower per row
                const int xb = g.x0 + seg * kSegOut;
                const bool edge = xb - 4 < 0 || xb + kSegOut + 4 > g.W;
                const int64_t work = (int64_t)((y1 - y0) + halo) * (edge ? p->edge_w4 : 4);
                items.push_back({i, seg, band, id, work});
                img_work[i] += work;
            }
        }
        if (items.size() > (size_t)(1 << 30)) { delete p; return SHINE_ERR_INVALID_ARG; }
        p->tile_begin.push_back((int)items.size());
    }
    p->ntiles = (int)items.size();
    // claim order: the persistent warps take the tiles in this order
    if (p->order == SHINE_ORDER_LONGEST_FIRST) {
        std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.work > b.work; });
    } else if (p->order == SHINE_ORDER_LARGEST_IMAGE_FIRST) {
        std::stable_sort(items.begin(), items.end(), [&](const Item& a, const Item& b) {
            return img_work[a.img] > img_work[b.img];
        });
    }  // SHINE_ORDER_IMAGE: image by image, band by band
    std::vector<int4> tiles(items.size());
    for (size_t t = 0; t < items.size(); ++t) tiles[t] = make_int4(items[t].img, items[t].seg, items[t].band, items[t].id);
    const size_t bytes_tiles = tiles.size() * sizeof(int4);
    const size_t bytes_br = (size_t)n * sizeof(int);
    const size_t off_br = (bytes_tiles + 255) / 256 * 256;
    const size_t off_tb = off_br + (bytes_br + 255) / 256 * 256;
    const size_t total = off_tb + (size_t)(n + 1) * sizeof(int);
    if (cudaMalloc(&p->dbuf, total) != cudaSuccess) { delete p; return cuda_status(cudaGetLastError()); }
    char* base = static_cast<char*>(p->dbuf);
    p->d_tiles = reinterpret_cast<int4*>(base);
    p->d_band_rows = reinterpret_cast<int*>(base + off_br);
    p->d_tile_begin = reinterpret_cast<int*>(base + off_tb);
    cudaError_t e = cudaMemcpy(p->d_tiles, tiles.data(), bytes_tiles, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_band_rows, p->band_rows.data(), bytes_br, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_tile_begin, p->tile_begin.data(), (size_t)(n + 1) * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(p->dbuf); delete p; return cuda_status(e); }
    p->grid = grid_for(dt, mode, p->staging);
    *plan = p;
    return SHINE_OK;
}

shine_status shine_plan_workspace(const shine_plan* plan, size_t* bytes) {
    if (!plan || !bytes) return SHINE_ERR_INVALID_ARG;
    *bytes = 256 + (size_t)kParamSlots * (size_t)plan->ntiles * sizeof(double);
    return SHINE_OK;
}

shine_status shine_plan_tile_rows(const shine_plan* plan, int32_t i, int32_t* rows) {
    if (!plan || !rows || i < 0 || i >= plan->n) return SHINE_ERR_INVALID_ARG;
    *rows = plan->band_rows[i];
    return SHINE_OK;
}

shine_status shine_plan_schedule(const shine_plan* plan, int32_t* order, int32_t* staging, int32_t* edge_w4,
                                 int32_t* origin) {
    if (!plan || !order || !staging || !edge_w4 || !origin) return SHINE_ERR_INVALID_ARG;
    *order = plan->order;
    *staging = plan->staging;
    *edge_w4 = plan->edge_w4;
    *origin = plan->origin;
    return SHINE_OK;
}

shine_status shine_pipeline_batched(const shine_plan* plan, const shine_image_desc* descs, const float* kappa,
                                    const float* wx, const float* wy, float* grad_kappa, float* grad_wx,
                                    float* grad_wy, void* workspace, size_t ws_bytes, void* stream) {
    SHINE_ENTRY("shine_pipeline_batched");
    if (!plan || !descs || !kappa || !wx || !wy) return SHINE_ERR_INVALID_ARG;
    size_t need = 0;
    shine_plan_workspace(plan, &need);
    if (!workspace || ws_bytes < need) return SHINE_ERR_WORKSPACE;
    if (!aligned_to(workspace, 256) || !aligned_to(descs, 8) || !aligned_to(kappa, 4)) return SHINE_ERR_ALIGNMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchArgs b;
    b.descs = descs;
    b.tiles = plan->d_tiles;
    b.band_rows = plan->d_band_rows;
    b.ntiles = plan->ntiles;
    b.n = plan->n;
    b.valid = plan->border == SHINE_VALID;
    b.origin = plan->origin;
    b.dbg = bounds_flag();
    // workspace header: the bounded-wait failure word (read by shine_workspace_status), then the
    // tile counter
    b.err = static_cast<unsigned int*>(workspace);
    b.counter = static_cast<unsigned int*>(workspace) + 1;
    b.partials = reinterpret_cast<double*>(static_cast<char*>(workspace) + 256);
    b.kappa = kappa; b.wx = wx; b.wy = wy;
    shine_status st = cuda_status(cudaMemsetAsync(workspace, 0, 2 * sizeof(unsigned int), s));
    if (st != SHINE_OK) return st;
    st = cuda_status(launch_batched(b, plan->dt, plan->mode, plan->staging, plan->grid, s));
    if (st != SHINE_OK) return st;
    if (plan->mode == SHINE_MODE_FWD_BWD && (grad_kappa || grad_wx || grad_wy)) {
        finalize_batched_kernel<<<plan->n + kParamSlots - 1, 256, 0, s>>>(b.partials, plan->ntiles, plan->n,
                                                                        plan->d_tile_begin, grad_kappa, grad_wx,
                                                                        grad_wy);
        st = cuda_status(cudaPeekAtLastError());
    }
    return st;
}

int shine_tune_key(char* buf, size_t len) {
    const std::string k = gpu_key();
    if (k == "unknown") return -1;
    if (buf && len > 0) {
        std::strncpy(buf, k.c_str(), len - 1);
        buf[len - 1] = '\0';
    }
    return (int)k.size();
}

void shine_plan_destroy(shine_plan* plan) {
    if (!plan) return;
    if (plan->dbuf) cudaFree(plan->dbuf);
    delete plan;
}

}  // extern "C"
