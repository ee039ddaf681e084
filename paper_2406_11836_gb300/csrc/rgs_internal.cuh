// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/rgs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rgs.h"

namespace rgs {

// ------------------------------------------------------------------ limits and layout
constexpr int kTile = 16;                 // tile edge (pixels)
constexpr int kTilePixels = kTile * kTile;
constexpr int kMaxRenderDepth = 6;        // K <= 64 subsets in a render (64-bit masks)
constexpr int kMaxKdDepth = 8;            // K <= 256 leaves in a partition
constexpr int kMaxNodes = (1 << kMaxKdDepth) - 1;

// Projected splat record: three float4 per splat (48 bytes), written by the projection
// and gathered by the blend kernels once per (tile, subset) instance.
//   r0 = (mean_x hi, mean_y hi, half2(mean_x lo, mean_y lo) bits, alpha)
//   r1 = (l11, l12, l22, rho2)   conic = L^T L with L = [[l11, l12], [0, l22]];
//                                rho2 = (D/z)^2, stored negated when the splat lies in
//                                more than one subset (the per-pixel Eq. 6 test is needed)
//   r2 = (r, g, b, z)
constexpr int kRecFloat4 = 3;

// Per-splat gradient record of the blend backward: 12 floats (three float4 so that
// accumulation can use vector reductions):
//   (mean_x, mean_y, conic_a, conic_b, conic_c, alpha, r, g, b, 0, 0, 0)
constexpr int kG2dFloats = 12;

// ------------------------------------------------------------------ kernel parameters
struct TreeParams {            // KD splits in heap order
    int L;
    int8_t axis[kMaxNodes];
    float split[kMaxNodes];
};

struct ViewParams {
    float R[9];                // world->camera rotation (row-major)
    float t[3];
    float o[3];                // camera centre (fp32 rounding of -R^T t)
    float fx, fy, cx, cy, ifx, ify, near_z;
    int W, H, tiles_x, tiles_y;
    float trunc_mult, eps_T, alpha_min, alpha_max, dilation;
    float bg[3];
    int K, L, sh_degree;
    int tile_bits;             // bits of the tile index in an instance key
    int8_t order[64];          // order[r]  = subset at view rank r
    int8_t rank_of[64];        // rank_of[k] = view rank of subset k
    // per-view plane templates of the KD leaves (see clip_table_kernel), [K * L] each:
    // device addresses, kept as 32-bit halves so that the struct stays 4-byte aligned (the
    // kernels' parameter layout, and with it their code, does not change)
    uint32_t clip_addr[4];
    __host__ __device__ const float4* clip_plane() const {
        return reinterpret_cast<const float4*>(((uint64_t)clip_addr[1] << 32) | clip_addr[0]);
    }
    __host__ __device__ const float* clip_margin() const {
        return reinterpret_cast<const float*>(((uint64_t)clip_addr[3] << 32) | clip_addr[2]);
    }
    __host__ void set_clip(const float4* plane, const float* margin) {
        clip_addr[0] = (uint32_t)(uintptr_t)plane;
        clip_addr[1] = (uint32_t)((uint64_t)(uintptr_t)plane >> 32);
        clip_addr[2] = (uint32_t)(uintptr_t)margin;
        clip_addr[3] = (uint32_t)((uint64_t)(uintptr_t)margin >> 32);
    }
    // 1: x_i is the foot of the perpendicular from the centre onto the pixel ray (the
    // comparison reading of Sec. 3.2, forward only); 0: the ray point at the splat's depth
    int foot;
    // 1: a subset is not blended on a ray whose merged transmittance in front of it is
    // below eps_T (rgs_render_opts::cull_occluded)
    int cull_occluded;
    // Binning by groups of view ranks (the image-only forward): count and emission take
    // only the subsets of rank in [bin_lo, bin_hi), and, when the open-tile table is set,
    // only the tiles it marks open: entry ty * (tiles_x + 1) + c holds the number of open
    // tiles among columns [0, c) of tile row ty.  fill_view sets every rank, no table.
    // With the open-tile table comes its summed-area table: entry y * (tiles_x + 1) + x
    // holds the open tiles in rows [0, y) and columns [0, x), so that a splat whose tile
    // box holds no open tile is passed over at once.
    int bin_lo, bin_hi;
    uint32_t open_addr[4];
    __host__ __device__ const uint32_t* open_prefix() const {
        return reinterpret_cast<const uint32_t*>(((uint64_t)open_addr[1] << 32) | open_addr[0]);
    }
    __host__ __device__ const uint32_t* open_sat() const {
        return reinterpret_cast<const uint32_t*>(((uint64_t)open_addr[3] << 32) | open_addr[2]);
    }
    __host__ void set_open(const uint32_t* table, const uint32_t* sat) {
        open_addr[0] = (uint32_t)(uintptr_t)table;
        open_addr[1] = (uint32_t)((uint64_t)(uintptr_t)table >> 32);
        open_addr[2] = (uint32_t)(uintptr_t)sat;
        open_addr[3] = (uint32_t)((uint64_t)(uintptr_t)sat >> 32);
    }
};
constexpr int kClipTable = 64 * kMaxRenderDepth;   // entries of one view's plane-template table

// ------------------------------------------------------------------ request batches (serve.cu)
// A batch renders up to kMaxSlots requests (views of the same resident scene) in one pass
// of device-counted kernels.  Per-splat arrays are indexed slot * N + i; tile indices are
// global over the batch: request s owns tiles [tile_base, tile_base + tiles_x * tiles_y).
constexpr int kMaxSlots = 16;

struct BatchSlot {
    ViewParams vp;
    float* image;              // [3, H, W] output of the request
    const float* grad;         // [3, H, W] dL/dimage (the batched backward; null in serving)
    uint32_t tile_base;        // first global tile of the request
    uint32_t state_base;       // first tile of its group state (binning in groups of view ranks)
};

struct BatchHeader {
    unsigned long long n_total;          // S * N: the projection's output domain
    int S;                               // requests in the batch
    uint32_t total_tiles;                // sum of the requests' tiles
    uint32_t tile_base[kMaxSlots + 1];   // prefix of the requests' tile counts
};

// One lane of batch buffers (serve.cu): the slot table and header the batch's kernels read,
// its device counters, each slot's plane templates, and the per-(slot, splat) and
// per-instance arrays.
struct LaneBufs;
// Device counters of a batch (uint64): [0] instances, [1] visible (slot, splat) pairs,
// [2] overflow flag, [3] blend work-queue head, [4] instances to sort (0 on overflow),
// [5], [6] emission work-queue heads, [7] the batched backward's work-queue head, then
// (instances, visible) per slot from kBatchSlotCounters, then the kept items.
constexpr int kBatchSlotCounters = 8;
// ... then the items the projection kept for the emission (one counter), then the
// projection candidates of each slot (their lists lie in vis_pos, slot s at s * N)
constexpr int kBatchItemCounter = kBatchSlotCounters + 2 * kMaxSlots;
constexpr int kBatchCandCounters = kBatchItemCounter + 1;
// ... then, binning in two groups of ranks: [0] the first group's instances, [1] the
// second's, [2] the second group's count work-queue head
constexpr int kBatchBinCounter = kBatchCandCounters + kMaxSlots;
constexpr int kBatchCounters = kBatchBinCounter + 3;

struct RasterBuffers;
int ceil_log2(int64_t x);

// Binning in two groups of view ranks (group_binning 1) pays when a render's tile
// instances average at least kGroupInstancesPerSplat per visible splat and number at least
// kGroupMinInstances: the later group's count and emission go over every visible splat
// (about 0.3 ns each on a GB300) and its extra passes cost about 0.2 ms, while each
// instance it spares the sort and the emission saves about 25 ps; in the views measured
// between a third and a half of the instances past the first group were left to bin.
constexpr int64_t kGroupInstancesPerSplat = 12;
constexpr int64_t kGroupMinInstances = (int64_t)1 << 24;

// ------------------------------------------------------------------ tracing
// Passes timed by the profiler (rgs_profile_*): a pair of CUDA events is recorded on the
// launching stream around each pass while profiling is on.
enum Stage {
    ST_PROJECT = 0, ST_COMPACT, ST_DEPTH_SORT, ST_OFFSETS, ST_EMIT, ST_INST_SORT, ST_RANGES, ST_BLEND_FWD,
    ST_BLEND_BWD, ST_PROJECT_BWD, ST_ADAM, ST_MERGE, ST_MERGE_BWD, ST_KD, ST_BATCH_FWD, ST_COUNT
};
struct ProfScope {
    int token;
    cudaStream_t s;
    ProfScope(int stage, cudaStream_t st);
    ~ProfScope();
};
// Device counters of evaluated / contributing (pixel, splat) pairs, or nullptr when
// profiling is off: [0] fwd evaluated, [1] fwd contributing, [2] bwd evaluated, [3] bwd
// contributing.
unsigned long long* prof_pair_counters();
void prof_add_host_counts(int64_t instances, int64_t visible);
void count_launch();   // every kernel launch of the library (reported with the tracing counters)
void prof_suppress(bool on);   // this thread's passes record no events while on

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
void set_required_workspace(size_t bytes);
// A value never seen before in this process (never 0): the stamp a forward writes into its
// workspace so that a backward can tell whether the lists there are still its own.
unsigned long long next_nonce();
// Streaming multiprocessors of the current device (queried once per device, cached); grid
// sizes of the grid-stride and persistent kernels are multiples of it.
int sm_count();

#define RGS_CUDA_TRY(expr)                                                                 \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess) {                                                           \
            ::rgs::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(_e)); \
            return RGS_ECUDA;                                                              \
        }                                                                                  \
    } while (0)

#define RGS_CUDA_LAUNCH_CHECK()                                                            \
    do {                                                                                   \
        ::rgs::count_launch();                                                             \
        cudaError_t _e = cudaGetLastError();                                               \
        if (_e != cudaSuccess) {                                                           \
            ::rgs::set_error("%s:%d: kernel launch: %s", __FILE__, __LINE__, cudaGetErrorString(_e)); \
            return RGS_ECUDA;                                                              \
        }                                                                                  \
    } while (0)

// ------------------------------------------------------------------ scan / sort (sort.cu)
// Exclusive prefix sum of n uint32 values; `in` may equal `out`.  `load` selects what
// is summed: 0 = the value, 1 = (value != 0), 2 = in[gather[i]].
size_t scan_temp_bytes(int64_t n);
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, int load, const uint32_t* gather, void* temp,
                       size_t temp_bytes, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on key bits [0, end_bit), 8-bit digits.
// The sorted pairs end in (keys, vals) or (keys_alt, vals_alt): *in_alt tells which.
size_t radix_temp_bytes(int64_t n);
int radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, int64_t n, int end_bit,
                     void* temp, size_t temp_bytes, cudaStream_t s, bool* in_alt);

// Device-counted variants: the element count is read on the device from *n_dev (clamped
// to cap, the buffers' capacity), so the launches need no host round trip and can be
// captured in a CUDA graph.  Fixed temporary sizes.
size_t scan_dev_temp_bytes();
int exclusive_scan_dev(const uint32_t* in, uint32_t* out, const unsigned long long* n_dev, int64_t cap, int load,
                       const uint32_t* gather, void* temp, size_t temp_bytes, cudaStream_t s);
size_t radix_dev_temp_bytes();
// Sets the wide sort passes' shared-memory attribute on the current device; call it before
// capturing a stream that sorts (the passes set it themselves outside a capture).
int sort_prepare();
int radix_sort_pairs_dev(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                         const unsigned long long* n_dev, int64_t cap, int end_bit, void* temp, size_t temp_bytes,
                         cudaStream_t s, bool* in_alt,
                         const unsigned long long* base_dev = nullptr);

// ------------------------------------------------------------------ raster (raster.cu)
struct RasterBuffers {
    // per splat
    float4* rec;          // [N * 3]
    uint32_t* cnt;        // [N] instances of the splat (0: culled)
    uint32_t* cnt_bin;    // [N] instances in the first binning group (nullptr: one group, cnt)
    unsigned long long* bin_ctr;    // their total
    // binning in groups of ranks (image-only forward)
    float4* state;        // [tiles * 256] each pixel's merged colour and front transmittance between groups
    uint8_t* open;        // [tiles] 1: a later group can still change the tile
    uint32_t* open_prefix;   // [tiles_y * (tiles_x + 1)] open tiles before each column, per tile row
    uint32_t* open_sat;      // [(tiles_y + 1) * (tiles_x + 1)] its summed-area table
    ushort4* rect;        // [N] tile rectangle (x0, y0, x1, y1), inclusive
    unsigned long long* mask;  // [N] subsets containing the splat
    uint32_t* dkey;       // [N] depth key (float bits of z)
    uint32_t* dkey_lo;    // [N] 16 bits of depth below the float z (depth_fraction)
    uint32_t* vis_pos;    // [N] compaction positions
    uint32_t* skey;       // [N] compacted depth keys   (sort buffer a)
    uint32_t* sid;        // [N] compacted splat ids     (sort buffer a)
    uint32_t* skey_alt;   // [N]                         (sort buffer b)
    uint32_t* sid_alt;    // [N]
    uint32_t* ioff;       // [N] instance offsets in depth order
    unsigned long long* counters;  // [16]: total instances, visible splats, -, -, emission work queues (2),
                                   // -, -, the splats each emission launch deferred (2), -, -,
                                   // items kept by the count (may exceed item_cap), projection
                                   // candidates (the list is in vis_pos until the compaction),
                                   // instances of the first binning group, of a later group
    uint32_t* item_at;    // [N] items kept by the count (footprint.cuh; nullptr: none kept)
    uint4* items;         // [item_cap] their records (first instance among the first binning group's)
    unsigned long long* item_ctr;   // records taken (may exceed item_cap)
    uint32_t* item_first_all;   // [item_cap] each kept item's first instance among all the splat's
    const uint32_t* item_first; // what the emission takes the items' first instances from
                                // (nullptr: the records; else item_first_all, one group)
    uint32_t* ibase;      // [N] first instance of each splat whose items were kept (set by the emission)
    uint32_t item_cap;
    uint4* units;         // per emission launch a list of unit_cap (id, instance base) pairs: the
                          // splats its first kernel defers to the second (nullptr: none deferred)
    uint32_t unit_cap;
    float4* g2d;          // [N * 3] (backward only)
    // per (tile, subset)
    uint2* ranges;        // [tiles * K]
    const float* cull;    // [tiles * K] forward depth table (backward only; nullptr: no culling)
    float2* cull_chunk;   // [tiles_y * ceil(tiles_x / 16) * K] (min, max) of `cull` over 16-tile chunks
    float4* clip_plane;   // [kClipTable] the view's plane templates (ViewParams::clip_plane())
    float* clip_margin;   // [kClipTable]
    unsigned long long* header;   // [32] workspace header: [0] the nonce of the forward whose lists it holds
    // foot reading only (nullptr otherwise)
    float4* foot_side;    // [N] ((D/z)^2, z lo, mx lo, my lo): the ball radius (the record carries +-inf so
                          // that no footprint uses it) and the low parts of the depth and centre
    uint32_t* fkey;       // [inst_cap] order-preserving bits of the per-(splat, tile) ray-parameter bound
    uint32_t* fidx;       // [inst_cap] instance positions
    // per instance
    uint32_t* ikey;
    uint32_t* ival;
    uint32_t* ikey_alt;
    uint32_t* ival_alt;
    int64_t inst_cap;
    // scratch for scans and sorts
    void* temp;
    size_t temp_bytes;
};

struct LaneBufs {
    unsigned long long* header;   // train layouts: [32] words, [0] the nonce of the forward whose lists it holds
    BatchSlot* slots;
    BatchHeader* hdr;
    unsigned long long* counters;
    float4* clip_plane;    // [kMaxSlots * kClipTable]: each request's plane templates
    float* clip_margin;    // [kMaxSlots * kClipTable]
    unsigned long long* one;   // a device word that is never 0 (the skip flag of unused slots)
    // binning in two groups of view ranks (serving lanes): the second group's slot table
    // (each request's view with its rank range and open-tile tables)
    BatchSlot* slots2;
    int64_t prefix_cap, sat_cap;   // entries of b.open_prefix / b.open_sat
    int64_t group_tiles;           // tiles of group state (b.state: 256 pixels each)
    RasterBuffers b;
};
// serve.cu: the lane layout (train: with 2D-gradient records) and the batch pipeline
// (projection of every (slot, splat) pair through the persistent blend, device-counted).
size_t lane_layout(char* base, int64_t N, int slots, int64_t tiles_cap, int K, int64_t inst_cap, LaneBufs* out,
                   bool train = false, int64_t group_tiles = 0);
// ival_out (nullable): the buffer that holds the sorted instance payloads.
// The per-request blend launches of a captured serving batch (graph nodes whose arguments
// each batch sets): first group (or every rank), second group; and the buffer that holds
// the sorted instance payloads.
struct BlendNodes {
    cudaGraphNode_t g1[kMaxSlots];
    cudaGraphNode_t g2[kMaxSlots];
    const uint32_t* ival;
};
// nodes (nullable): blend each request by its own launch (recorded in *nodes) instead of
// the persistent batch blend.  grouped (slots2_host set; needs nodes and a lane laid out
// with group state): the slots bin view ranks [0, bin_hi) first, and those of slots2 ranks
// [bin_lo, K) in the tiles the first group left open.
int enqueue_batch(const rgs_gaussians& g, const TreeParams& tp, int K, int L, int slots, int64_t tiles_cap,
                  const LaneBufs& l, const BatchSlot* slots_host, const BatchHeader* hdr_host,
                  unsigned long long* status_host, cudaStream_t s, bool record_ends = false,
                  const uint32_t** ival_out = nullptr, const BatchSlot* slots2_host = nullptr,
                  BlendNodes* nodes = nullptr);

int launch_project_fwd(const rgs_gaussians& g, const ViewParams& vp, const TreeParams& tp, RasterBuffers& b,
                       cudaStream_t s);
// Fills vp.clip_plane / vp.clip_margin (device) for one view, or for every slot of a batch
// (each slot's view carries its own table pointers).
int launch_clip_table(const ViewParams& vp, const TreeParams& tp, cudaStream_t s);
int launch_clip_table_batch(const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp, cudaStream_t s);
int launch_project_bwd(const rgs_gaussians& g, const rgs_gaussian_grads& gr, const ViewParams& vp,
                       const RasterBuffers& b, cudaStream_t s);
int launch_project_batch(const rgs_gaussians& g, const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp,
                         const RasterBuffers& b, unsigned long long* counters, cudaStream_t s);
// Batch emission over the (slot, depth)-sorted visible list (count counters[1]); writes
// nothing when the overflow flag counters[2] is set.
// inst_base (nullable): the instances start at that index (a device value); open_tables:
// the slots' views carry open-tile tables (a later binning group).
int launch_emit_batch(const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp, const RasterBuffers& b,
                      const uint32_t* sorted_ids, int64_t n_cap, int64_t N, unsigned long long* counters,
                      cudaStream_t s, const unsigned long long* inst_base = nullptr, bool open_tables = false);
// A later binning group of a batch: each slot's open-tile tables from the open flags (at
// the addresses its view carries).
int launch_open_tables_batch(const BatchSlot* slots, const BatchHeader* hdr, const uint8_t* open, cudaStream_t s);
// ... and its count for every visible (slot, splat) pair in depth order (into cnt_out;
// total into *total), as launch_recount.
int launch_recount_batch(const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp, const RasterBuffers& b,
                         const uint32_t* sorted_ids, int64_t n_cap, int64_t N, unsigned long long* counters,
                         uint32_t* cnt_out, unsigned long long* queue, unsigned long long* total, cudaStream_t s);
int launch_ranges_dev(const uint32_t* keys, const unsigned long long* n_dev, int64_t cap, uint2* ranges,
                      cudaStream_t s, const unsigned long long* base_dev = nullptr);
// Persistent forward blend over the batch's global tiles (fused merge into each slot's
// image; no partial maps).  record_ends: cut each saturated run back to what was staged
// (the batched backward replays the runs).
// One request of a serving batch blended by its own launch of the forward blend kernel
// (view ranks [r_begin, r_end), its tiles' ranges, group state and open flags, its image;
// nothing when *skip is set): launched while a lane's graph is captured, its graph node
// then given each batch's arguments and grid (the request's tiles).
struct BlendNodeArgs {
    ViewParams vp;
    TreeParams tp;
    uint2* ranges;
    const uint32_t* ival;
    const float4* rec;
    float* image;
    int r_begin, r_end;
    float4* state;
    uint8_t* open;
    const unsigned long long* skip;
};
int launch_blend_node(const BlendNodeArgs& a, unsigned grid, cudaStream_t s);
int set_blend_node(cudaGraphExec_t exec, cudaGraphNode_t node, const BlendNodeArgs& a, unsigned grid);
int launch_blend_batch(const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp, uint2* ranges,
                       const uint32_t* ival, const float4* rec, unsigned long long* counters, cudaStream_t s,
                       bool record_ends = false);
// Persistent flat backward over the batch's global tiles (counters[7]: its work queue);
// 2D gradients into g2d indexed like rec (slot * N + splat).
int launch_blend_bwd_batch(const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp, const uint2* ranges,
                           const uint32_t* ival, const float4* rec, float4* g2d, int64_t n_inst, int64_t n_splats,
                           unsigned long long* counters, cudaStream_t s);
int launch_emit(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* sorted_ids,
                int64_t n_vis, cudaStream_t s);
// first: the index of keys[0] in the whole instance array; clear: zero the table first.
int launch_ranges(const uint32_t* keys, int64_t n, uint2* ranges, int64_t n_ranges, cudaStream_t s,
                  uint32_t first = 0, bool clear = true);
// Binning in groups of ranks: the open-tile tables from the per-tile flags, and the count of
// a later group (vp's rank range and open-tile table) per visible splat in depth order
// (rewrites the kept items' offsets for that group; counters[4] is its work queue and
// counters[15] its total, both zeroed by the caller).
int launch_open_prefix(const ViewParams& vp, const uint8_t* open, uint32_t* prefix, uint32_t* sat, cudaStream_t s);
int launch_recount(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* sorted_ids,
                   int64_t n_vis, uint32_t* cnt_out, cudaStream_t s);
int launch_cull_chunks(const ViewParams& vp, const float* cull, float2* chunk, cudaStream_t s);
// record_ends: where a subset saturates a tile, b.ranges' end is moved back to the end of
// the last batch the blend staged (the prefix a backward has to replay).
// r_begin, r_end: the view ranks blended (r_end < 0: to K); a group other than the whole
// range needs an image-only render and b.state / b.open (blend_fwd_tile).
int launch_blend_fwd(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* ival,
                     float* partial_C, float* partial_T, float* image, float* T_final, float* tile_depth,
                     cudaStream_t s, bool record_ends = false, int r_begin = 0, int r_end = -1);
// Foot reading (forward only): orders the emitted instances by (tile, subset, bound of
// the foot's ray parameter over the tile) and returns the sorted keys and payloads.
int launch_foot_order(const ViewParams& vp, const RasterBuffers& b, int64_t I, cudaStream_t s,
                      const uint32_t** keys_out, const uint32_t** vals_out);
// Foot-reading forward blend; `over` (device, zeroed by the caller) counts pending-buffer overflows.
int launch_blend_foot(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* ival,
                      float* partial_C, float* partial_T, float* image, float* T_final,
                      unsigned long long* over, cudaStream_t s);
// Its backward (flat form): adds each blended pair's 2D gradients to b.g2d (zeroed by the
// caller); image is the forward's, dL_dimage [3,H,W]; `over` as above.
int launch_blend_foot_bwd(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* ival,
                          const float* image, const float* dL_dimage, unsigned long long* over, cudaStream_t s);
// n_inst: instances in ival (ranges are clamped to it); n_splats: records in b.rec (other
// payloads are skipped).  image != nullptr: the flat form (from the merged image; the
// partial maps are not read), else the per-subset form from the partial maps.
int launch_blend_bwd(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* ival,
                     const float* partial_C, const float* partial_T, const float* image, const float* dL_dimage,
                     int64_t n_inst, int64_t n_splats, cudaStream_t s);
int launch_merge(const float* pC, const float* pT, const int32_t* order, int K, int H, int W, const float bg[3],
                 float* image, float* T_out, cudaStream_t s);
int launch_merge_bwd(const float* pC, const float* pT, const int32_t* order, int K, int H, int W, const float bg[3],
                     const float* gI, const float* gT, float* dC, float* dT, cudaStream_t s);

// Forward render into a caller-given workspace.  host_counters (2 x uint64, nullable)
// receives the instance and visible-splat counts; NULL uses a pinned buffer of the library.
// keep_lists: with partial maps, register the workspace's lists for the backward of this
// render (a host-side table entry; false for callers that must not allocate).
int render_fwd_into(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
                    float* partial_C, float* partial_T, float* image, float* T_final, float* tile_depth,
                    void* workspace, size_t ws_bytes, cudaStream_t s, unsigned long long* host_counters,
                    bool keep_lists = true);

// ------------------------------------------------------------------ KD (kd.cu)
struct KdBuild {
    int L;
    int8_t axis[kMaxNodes];
    float split[kMaxNodes];
    int64_t offsets[(1 << kMaxKdDepth) + 1];
    int32_t* idx_dev;   // cudaMalloc'd, M entries
    int64_t M;
};
int kd_build(const rgs_gaussians& g, int L, float trunc_mult, KdBuild* out, cudaStream_t s);
// Subset lists N_k for the splits already in `out` (out->L, axis, split).
int kd_subsets(const rgs_gaussians& g, float trunc_mult, KdBuild* out, cudaStream_t s);

// ------------------------------------------------------------------ argument checks and view setup (abi.cu)
bool aligned(const void* p, size_t a);
size_t a256(size_t x);
int check_gaussians(const rgs_gaussians* g);
int check_camera(const rgs_camera* c);
int check_opts(const rgs_render_opts* o);
void view_order_host(const struct ::rgs_kd* kd, const rgs_camera* cam, int32_t* order);
void fill_view(const struct ::rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
               ViewParams* vp, TreeParams* tp);

// ------------------------------------------------------------------ Adam (adam.cu)
// pseg >= 0: inside segment pseg, elements whose offset from the segment start is below
// `head` modulo `period` take head_lr.
int launch_adam(float* p, float* g, float* m, float* v, int64_t n, const int64_t* seg_off, const float* seg_lr,
                int nseg, float b1, float b2, float eps, float bc1, float bc2, int zero_grad, cudaStream_t s,
                int pseg = -1, int64_t period = 1, int64_t head = 0, float head_lr = 0.f);

}  // namespace rgs

// ------------------------------------------------------------------ opaque handles
struct rgs_kd {
    rgs::KdBuild b;
    int device;
    float trunc_mult;
};
