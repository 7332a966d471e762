// Host-visible launch descriptors of the Harris kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace shine {

constexpr int kCols = 4;                       // pixels per lane
constexpr int kLanes = 32;
constexpr int kSegLoad = kLanes * kCols;       // 128 staged columns per warp segment
constexpr int kSegOut = (kLanes - 2) * kCols;  // 120 computed columns per warp segment
// Compile-time tuning of the kernels (each has a default; the values are chosen by measurement).
#ifndef SHINE_FWD_STAGES
#define SHINE_FWD_STAGES 2        // image rows the forward keeps in flight (register staging)
#endif
#ifndef SHINE_FWD_EDGE_STAGES
#define SHINE_FWD_EDGE_STAGES 1   // the same on edge segments (fewer rows: less code next to the
#endif                            // bulk-staged strips; measured 7% faster forward)
#ifndef SHINE_FWD_TMA
#define SHINE_FWD_TMA 1           // forward interior segments staged by bulk copies
#endif
#ifndef SHINE_FWD_BULK_STAGES
#define SHINE_FWD_BULK_STAGES 4   // shared-memory slots of the forward's bulk staging ring
#endif
#ifndef SHINE_FWD_MIN_BLOCKS
#define SHINE_FWD_MIN_BLOCKS 4    // resident CTAs per SM the forward register budget must allow
#endif
#ifndef SHINE_BWD_STAGES
#define SHINE_BWD_STAGES 8        // staged rows of the backward ring
#endif
#ifndef SHINE_BWD_TMA
#define SHINE_BWD_TMA 1           // backward interior segments staged by bulk copies
#endif
#ifndef SHINE_WIDE_BWD
#define SHINE_WIDE_BWD 1          // adjoint of aligned 16-bit CLAMP images: eight columns per lane
#endif
#ifndef SHINE_WIDE_BWD_STAGES
#define SHINE_WIDE_BWD_STAGES 4   // its staging ring (rows)
#endif
#ifndef SHINE_WIDE_BWD_F32
#define SHINE_WIDE_BWD_F32 0      // float32 images take it too
#endif
#ifndef SHINE_WIDE_BWD_STAGES_F32
#define SHINE_WIDE_BWD_STAGES_F32 3  // its staging ring for float32 images (8 warps x 28 KB)
#endif
#ifndef SHINE_WIDE_BWD_FUSED
#define SHINE_WIDE_BWD_FUSED 1    // the fused forward+backward pass of those images takes it too
#endif
#ifndef SHINE_WIDE_BWD_MIN_PIXELS
#define SHINE_WIDE_BWD_MIN_PIXELS (int64_t(1) << 25)  // smaller images keep the four-column adjoint
#endif
#ifndef SHINE_WIDE_BWD_SWAP_PAIRS
#define SHINE_WIDE_BWD_SWAP_PAIRS 1  // conflict-free float32 reads of the staged pieces
#endif
#ifndef SHINE_WIDE_BWD_ORIGIN
#define SHINE_WIDE_BWD_ORIGIN 0   // first output column of its segment 0 (a multiple of 8)
#endif
static_assert(SHINE_WIDE_BWD_ORIGIN % 8 == 0 && SHINE_WIDE_BWD_ORIGIN > -240 && SHINE_WIDE_BWD_ORIGIN <= 0,
              "the eight-column adjoint needs whole lanes inside or outside the image");
#ifndef SHINE_WIDE_BWD_EDGE_WEIGHT4
#define SHINE_WIDE_BWD_EDGE_WEIGHT4 8  // an edge-segment row weighs this / 4 interior rows (measured:
#endif                              // 8 best of 6, 8, 10 on 8192^2 bf16)
#ifndef SHINE_FWD_EDGE_WEIGHT4
#define SHINE_FWD_EDGE_WEIGHT4 6  // an edge-segment row weighs this / 4 interior rows (forward-type)
#endif
#ifndef SHINE_BWD_EDGE_WEIGHT4
#define SHINE_BWD_EDGE_WEIGHT4 6  // the same for the adjoint
#endif
#ifndef SHINE_FWD_BAND_MAJOR
#define SHINE_FWD_BAND_MAJOR 1    // forward: equal row bands across all segments
#endif
#ifndef SHINE_BWD_BAND_MAJOR
#define SHINE_BWD_BAND_MAJOR 0    // backward: even segment-major slices
#endif
constexpr int kFwdThreads = 128;  // 4 warps per CTA
constexpr int kFwdStages = SHINE_FWD_STAGES;
constexpr int kFwdEdgeStages = SHINE_FWD_EDGE_STAGES;
constexpr int kFwdBulkStages = SHINE_FWD_BULK_STAGES;
constexpr int kBwdThreads = 128;
constexpr int kBwdStages = SHINE_BWD_STAGES;
#ifndef SHINE_BWD_STAGES_F32
#define SHINE_BWD_STAGES_F32 7    // the single-image adjoint's ring for float32 images (measured:
#endif                            // 7 rows 0.426 ms, 5 0.433, 6 0.431, 8 0.432 on 8192^2)
template <typename TI> constexpr int bwd_stages() { return sizeof(TI) == 4 ? SHINE_BWD_STAGES_F32 : kBwdStages; }

constexpr int kParamSlots = 19;   // d kappa, d Wx[9], d Wy[9]

// Geometry shared by all kernels: which output region of the image a launch covers and how
// it is cut into (column segment, row band) work items of one warp each.
struct Geometry {
    int H, W;          // image size
    int valid;         // 1: VALID borders (output (H-4)x(W-4)), 0: CLAMP (output HxW)
    int xlo, xhi;      // output columns, in image coordinates: [xlo, xhi)
    int ylo, yhi;      // output rows, in image coordinates: [ylo, yhi)
    int ox, oy;        // image coordinates of output element (0, 0)
    int x0;            // first output column of segment 0 (image coordinates)
    int nseg;          // column segments of kSegOut output columns
    int nband, band_rows;  // row bands (tile lists of the batched path)
    int nwarps;        // single-image kernels: warps sharing the nseg x rows work units
    unsigned int* dbg; // debug builds: the index-check violation word (null otherwise)
};

// Debug builds (compiled with SHINE_DEBUG_BOUNDS=1, the library libshine_debug.so) check the index
// ranges of the Harris kernels' global loads, stores and copies and of their shared-memory
// staging against the image, output and ring extents, and on a violation set bit `bit` of the
// violation word (no trap; the access still happens as it would in a release build, so a debug
// run gives the release results). Release builds compile the checks away.
#ifndef SHINE_DEBUG_BOUNDS
#define SHINE_DEBUG_BOUNDS 0
#endif
enum : int {
    kDbgFwdLoad = 0,     // forward: image row or column range of a vector load
    kDbgFwdStore = 1,    // forward: output row or column range of a store
    kDbgFwdStage = 2,    // forward: bulk copy or per-lane copy source range
    kDbgBwdStage = 3,    // adjoint: image or cotangent copy source range
    kDbgBwdStore = 4,    // adjoint: d img or R store range
    kDbgSmem = 5,        // a staging access outside the CTA's dynamic shared memory
};
#define SHINE_CHECK(dbgp, cond, bit)                                           \
    do {                                                                       \
        if constexpr (SHINE_DEBUG_BOUNDS) {                                    \
            if (!(cond) && (dbgp) != nullptr) atomicOr((dbgp), 1u << (bit));   \
        }                                                                      \
    } while (0)

// Balanced split of n work units over t workers: worker w gets [lo, hi), sizes differ by <= 1.
__host__ __device__ inline void balanced_slice(int64_t n, int64_t t, int64_t w, int64_t& lo, int64_t& hi) {
    const int64_t q = n / t, rem = n % t;
    lo = q * w + (w < rem ? w : rem);
    hi = lo + q + (w < rem ? 1 : 0);
}

// Work of warp w among t warps over nseg segments x rows rows, as (segment, row) units in
// segment-major order: [lo, hi). The two edge segments (first and last) run slower per row than
// the interior ones (element staging, clamps), so a unit of theirs weighs ew4 / 4 interior units
// (ew4 = 4: no weighting); every warp gets about the same weight, so that no edge warp is left
// running alone at the end.
// Band-major: when t >= nseg, every warp takes one segment and one row band of it; the warps of
// one interior band walk the same rows at the same time (whole image rows, good DRAM page
// locality); edge segments are cut into proportionally more bands. Otherwise the weighted units
// are split evenly in segment-major order.
__host__ __device__ inline void warp_work(bool band_major, int64_t nseg, int64_t rows, int64_t t, int64_t w,
                                          int64_t& lo, int64_t& hi, int ew4 = 4) {
    const bool weigh = ew4 != 4 && nseg >= 3;
    if (band_major && t >= nseg) {
        if (!weigh) {
            const int64_t nb = t / nseg;
            if (w >= nb * nseg) { lo = hi = 0; return; }
            const int64_t seg = w % nseg, band = w / nseg;
            int64_t r0, r1;
            balanced_slice(rows, nb, band, r0, r1);
            lo = seg * rows + r0;
            hi = seg * rows + r1;
            return;
        }
        // bands per interior segment nbi and per edge segment nbe ~ nbi * ew4 / 4
        int64_t nbi = (4 * t) / (4 * (nseg - 2) + 2 * ew4);
        if (nbi < 1) nbi = 1;
        int64_t nbe = (nbi * ew4 + 2) / 4;
        const int64_t spare = (t - (nseg - 2) * nbi) / 2;
        if (nbe > spare) nbe = spare;
        if (nbe < 1) nbe = 1;
        if (nbe > rows) nbe = rows;
        if (nbi > rows) nbi = rows;
        int64_t seg, band, nb;
        if (w < 2 * nbe) {
            seg = w < nbe ? 0 : nseg - 1;
            band = w < nbe ? w : w - nbe;
            nb = nbe;
        } else {
            const int64_t v = w - 2 * nbe;
            if (v >= (nseg - 2) * nbi) { lo = hi = 0; return; }
            seg = 1 + v % (nseg - 2);
            band = v / (nseg - 2);
            nb = nbi;
        }
        int64_t r0, r1;
        balanced_slice(rows, nb, band, r0, r1);
        lo = seg * rows + r0;
        hi = seg * rows + r1;
        return;
    }
    if (!weigh) {
        balanced_slice(nseg * rows, t, w, lo, hi);
        return;
    }
    // weight positions: edge segment 0 | interior segments | edge segment nseg-1
    const int64_t e0 = rows * ew4, mid = (nseg - 2) * rows * 4, total = 2 * e0 + mid;
    auto unit = [&](int64_t p) -> int64_t {
        if (p < e0) return p / ew4;
        if (p < e0 + mid) return rows + (p - e0) / 4;
        return (nseg - 1) * rows + (p - e0 - mid) / ew4;
    };
    int64_t p0, p1;
    balanced_slice(total, t, w, p0, p1);
    lo = unit(p0);
    hi = p1 >= total ? nseg * rows : unit(p1);
}

struct FwdArgs : Geometry {
    const void* img;
    int64_t img_pitch;  // elements
    void* out;
    int64_t out_pitch;  // elements
    const float* kappa;
    const float* wx;
    const float* wy;
    int aligned;  // image rows can be staged with 16 / 8-byte copies
    int out_vec;  // output rows can be written with 16-byte vector stores
    int tma;      // interior segments may use bulk (TMA) staging (16-byte aligned rows)
    unsigned int* err;  // nonzero after a bounded wait gave up (nullable)
};

// Corner detection: the forward pass plus threshold and 3x3 non-maximum suppression of R.
// f.out (R) may be null; the mask is one byte per output pixel.
struct CornerArgs {
    FwdArgs f;
    uint8_t* mask;
    int64_t mask_pitch;  // bytes
    float threshold;
    int mask_vec;        // mask rows can be written 8 bytes at a time
};

// The backward pass always covers every image pixel (its output is d img, H x W), so its
// Geometry is the full image; the cotangent grad_out sits at (oy, ox) inside it with size
// (gho, gwo) (VALID: offset 2 and size (H-4, W-4); CLAMP: offset 0 and size (H, W)).
struct BwdArgs : Geometry {
    const void* img;
    int64_t img_pitch;
    const void* gout;
    int64_t gout_pitch;
    int gho, gwo;
    void* gimg;        // nullable
    int64_t gimg_pitch;
    const float* kappa;
    const float* wx;
    const float* wy;
    double* partials;  // slot i of warp w at partials[i * pstride + poffset + w]
    int64_t pstride;   // 0: nwarps (one launch owns the partials)
    int64_t poffset;
    unsigned int* err; // nonzero after a bounded wait gave up (reset by the host before launch)
    int tma;           // interior segments may use bulk (TMA) staging
    int aligned;       // image staging
    int g_aligned;     // cotangent staging (CLAMP with aligned pointer and pitch)
    int gimg_vec;      // d img rows can be written with vector stores (16 / 8-byte aligned rows; the
                       // eight-column kernel needs 16 for every storage type)
    void* rout;        // fused forward output R (nullable; storage type of the image)
    int64_t rout_pitch;
    int rout_vec;      // R rows can be written with 16 / 8-byte stores
};

// The launchers choose a.nwarps: one resident wave (occupancy x SMs), at most max_warps, and
// no more than leaves each warp min_rows rows. The backward's partials need
// kParamSlots x a.nwarps doubles; *nwarps_used (nullable) reports the count.
cudaError_t launch_harris_fwd(FwdArgs a, int dt, int out_dt, cudaStream_t s);
cudaError_t launch_harris_corners(CornerArgs c, int dt, int out_dt, cudaStream_t s);
cudaError_t launch_harris_bwd(BwdArgs a, int dt, int gout_dt, int max_warps, cudaStream_t s, int* nwarps_used);
// Minimum rows per warp slice when an image has fewer (segment, row) units than resident warps:
// small images take more, shorter slices (measured, L2 flushed: 512^2 forward 16.4 -> 10.2 us,
// adjoint 54 -> 34 us; 1024^2 adjoint 52 -> 40 us; 8192^2 unchanged).
#ifndef SHINE_FWD_MIN_ROWS
#define SHINE_FWD_MIN_ROWS 2
#endif
#ifndef SHINE_BWD_MIN_ROWS
#define SHINE_BWD_MIN_ROWS 4
#endif
constexpr int kFwdMinRows = SHINE_FWD_MIN_ROWS;
constexpr int kBwdMinRows = SHINE_BWD_MIN_ROWS;
constexpr int kMaxWarpsPerSm = 64;
constexpr size_t kWorkspaceHeader = 256;  // backward workspace: error word, then the partial sums
// First output column of segment 0 in the single-image kernels, per pass. Any origin = 4
// (mod 8) makes every interior segment's staged span (4 columns left of its output) start on
// an 8-pixel boundary, i.e. a 16-byte boundary for float32 and 16-bit rows and cotangents alike,
// which bulk copies require. Which of them is fastest depends on how the spans fall on the
// memory system; chosen by sweeps of -116 .. -12 on 2048^2 .. 8192^2 (forward: -108, 11% faster than
// -116 in bf16, equal in float32; adjoint: -76, 1-2% faster).
#ifndef SHINE_FWD_SEGMENT_ORIGIN
#define SHINE_FWD_SEGMENT_ORIGIN -108
#endif
#ifndef SHINE_BWD_SEGMENT_ORIGIN
#define SHINE_BWD_SEGMENT_ORIGIN -76
#endif
// First output column of segment 0 in the forward kernel, whose segments are 240 output columns
// wide (8 per lane), per storage type: any multiple of 8 in (-240, 0] makes every interior
// segment's staged span (8 columns left of its output) start on a 16-byte boundary for float32
// and 16-bit rows.
#ifndef SHINE_WIDE_ORIGIN_F32
#define SHINE_WIDE_ORIGIN_F32 -232
#endif
#ifndef SHINE_WIDE_ORIGIN_16
#define SHINE_WIDE_ORIGIN_16 0
#endif
template <typename TI> constexpr int wide_origin() { return sizeof(TI) == 4 ? SHINE_WIDE_ORIGIN_F32 : SHINE_WIDE_ORIGIN_16; }
static_assert(SHINE_WIDE_ORIGIN_F32 % 8 == 0 && SHINE_WIDE_ORIGIN_F32 > -240 && SHINE_WIDE_ORIGIN_F32 <= 0 &&
              SHINE_WIDE_ORIGIN_16 % 8 == 0 && SHINE_WIDE_ORIGIN_16 > -240 && SHINE_WIDE_ORIGIN_16 <= 0,
              "wide segment spans must start on 8-pixel boundaries");
// Shared-memory slots of the forward's bulk staging ring (measured on 8192^2 float32: 4 slots
// 0.173 ms, 6 slots 0.185 ms).
#ifndef SHINE_WIDE_CORNERS_MIN_BLOCKS
#define SHINE_WIDE_CORNERS_MIN_BLOCKS 3  // the corner kernel: resident 128-thread CTAs per SM (registers)
#endif
#ifndef SHINE_WIDE_BULK_STAGES
#define SHINE_WIDE_BULK_STAGES 4
#endif
// Edge segments of bulk-staged forward kernels: 1 = per-lane cp.async into the shared-memory ring,
// 0 = registers with L2 prefetch.
#ifndef SHINE_WIDE_EDGE_LANES
#define SHINE_WIDE_EDGE_LANES 1
#endif
// Forward staging of interior segments per storage type: 1 = bulk copies into a shared-memory
// ring, 0 = registers one row ahead with an L2 bulk prefetch kPfRows ahead (edge segments always
// use the latter).
#ifndef SHINE_WIDE_BULK_F32
#define SHINE_WIDE_BULK_F32 1
#endif
#ifndef SHINE_WIDE_BULK_16
#define SHINE_WIDE_BULK_16 0
#endif
#ifndef SHINE_WIDE_PF_ROWS
#define SHINE_WIDE_PF_ROWS 4
#endif
constexpr int kWidePfRows = SHINE_WIDE_PF_ROWS;
// Resident CTAs per SM the forward kernel's register budget must allow (3: 168 registers, 12
// warps per SM).
#ifndef SHINE_WIDE_MIN_BLOCKS
#define SHINE_WIDE_MIN_BLOCKS 3
#endif
constexpr int kFwdSegmentOrigin = SHINE_FWD_SEGMENT_ORIGIN;
constexpr int kBwdSegmentOrigin = SHINE_BWD_SEGMENT_ORIGIN;
static_assert(((kFwdSegmentOrigin % 8) + 8) % 8 == 4 && ((kBwdSegmentOrigin % 8) + 8) % 8 == 4,
              "segment spans must start on 8-pixel boundaries");
static_assert(kFwdSegmentOrigin > -120 && kBwdSegmentOrigin > -120, "segment 0 must reach column 0");
// out[f] = sum over n partials[f * n + i] (fixed order, float64), f < kParamSlots; any out
// pointer may be NULL.
cudaError_t launch_finalize_params(const double* partials, int64_t n, float* gkappa, float* gwx,
                                   float* gwy, cudaStream_t s);

}  // namespace shine
