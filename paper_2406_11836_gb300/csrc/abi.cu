// C ABI of the library (include/rgs.h): argument checks, workspace layout and the order
// of the passes of a render.  All arithmetic of the method runs in the kernels of
// project.cu, raster.cu, sort.cu, kd.cu and adam.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "rgs_internal.cuh"


namespace rgs {

// ------------------------------------------------------------------ errors
namespace {
thread_local char g_err[512] = "";
thread_local size_t g_required = 0;
}  // namespace

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}
void set_required_workspace(size_t bytes) { g_required = bytes; }

namespace {
constexpr int kMaxSmCache = 64;
std::atomic<int> g_sms[kMaxSmCache];   // 0: not queried yet
}  // namespace

int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    int n = dev >= 0 && dev < kMaxSmCache ? g_sms[dev].load(std::memory_order_relaxed) : 0;
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    if (dev >= 0 && dev < kMaxSmCache) g_sms[dev].store(n, std::memory_order_relaxed);
    return n;
}

// ------------------------------------------------------------------ profiler
namespace {
const char* kStageNames[ST_COUNT] = {"project", "compact", "depth_sort", "offsets", "emit", "instance_sort", "ranges",
                                     "blend_fwd", "blend_bwd", "project_bwd", "adam", "merge", "merge_bwd", "kd",
                                     "batch_fwd"};
struct Profiler {
    std::mutex mu;
    bool on = false;      // stage timing
    bool count = false;   // pair counters (counting kernel variants)
    std::vector<cudaEvent_t> pool;
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> open;      // started, not yet ended (indexed by token)
    std::vector<Rec> done;
    double ms[ST_COUNT] = {};
    int64_t launches[ST_COUNT] = {};
    int64_t host_counts[2] = {};
    unsigned long long* dev_pairs = nullptr;
    cudaEvent_t take() {
        if (pool.empty()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
};
Profiler g_prof;
}  // namespace

namespace {
thread_local bool g_prof_suppress = false;   // set only while a render must not create events
}
void prof_suppress(bool on) { g_prof_suppress = on; }

ProfScope::ProfScope(int stage, cudaStream_t st) : token(-1), s(st) {
    if (g_prof_suppress) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (!g_prof.on) return;
    Profiler::Rec r{stage, g_prof.take(), g_prof.take()};
    cudaEventRecord(r.a, s);
    g_prof.open.push_back(r);
    token = (int)g_prof.open.size() - 1;
}

ProfScope::~ProfScope() {
    if (token < 0) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (token >= (int)g_prof.open.size()) return;
    Profiler::Rec r = g_prof.open[token];
    cudaEventRecord(r.b, s);
    g_prof.done.push_back(r);
    if (token == (int)g_prof.open.size() - 1) g_prof.open.pop_back();
    else g_prof.open[token].stage = -1;
    while (!g_prof.open.empty() && g_prof.open.back().stage < 0) g_prof.open.pop_back();
}

unsigned long long* prof_pair_counters() { return g_prof.count ? g_prof.dev_pairs : nullptr; }

namespace {
std::atomic<int64_t> g_launches{0};
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void prof_add_host_counts(int64_t instances, int64_t visible) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (!g_prof.on && !g_prof.count) return;
    g_prof.host_counts[0] += instances;
    g_prof.host_counts[1] += visible;
}

namespace {

__global__ void compact_kernel(const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ pos,
                               const uint32_t* __restrict__ dkey_lo, int64_t n, uint32_t* __restrict__ skey,
                               uint32_t* __restrict__ sid) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || cnt[i] == 0) return;
    uint32_t p = pos[i];
    skey[p] = dkey_lo[i];
    sid[p] = (uint32_t)i;
}

__global__ void store_u64_kernel(unsigned long long* p, unsigned long long v) { *p = v; }

// key[j] = dkey[id[j]]: the float bits of z in the order of the first (low-bits) pass.
__global__ void gather_key_kernel(const uint32_t* __restrict__ dkey, const uint32_t* __restrict__ id, int64_t n,
                                  uint32_t* __restrict__ key) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) key[j] = dkey[id[j]];
}

}  // namespace

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

int check_gaussians(const rgs_gaussians* g) {
    if (!g) { set_error("gaussians: NULL"); return RGS_EINVAL; }
    if (g->n < 1 || g->n > 0x7fffffffll) { set_error("gaussians: n = %lld out of range [1, 2^31)", (long long)g->n); return RGS_EINVAL; }
    if (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh) {
        set_error("gaussians: NULL parameter pointer");
        return RGS_EINVAL;
    }
    if (g->sh_degree < 0 || g->sh_degree > 3) { set_error("gaussians: sh_degree %d not in 0..3", g->sh_degree); return RGS_EINVAL; }
    if (!aligned(g->quats, 16) || !aligned(g->means, 4) || !aligned(g->log_scales, 4) || !aligned(g->sh, 4) ||
        !aligned(g->opacity_logits, 4)) {
        set_error("gaussians: misaligned pointer (quats must be 16-byte aligned)");
        return RGS_EINVAL;
    }
    return RGS_OK;
}

int check_camera(const rgs_camera* c) {
    if (!c) { set_error("camera: NULL"); return RGS_EINVAL; }
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(c->viewmat[i])) { set_error("camera: non-finite view matrix"); return RGS_EINVAL; }
    if (!(std::isfinite(c->fx) && std::isfinite(c->fy) && std::isfinite(c->cx) && std::isfinite(c->cy) && c->fx > 0 &&
          c->fy > 0)) {
        set_error("camera: invalid intrinsics");
        return RGS_EINVAL;
    }
    if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384) {
        set_error("camera: image size %dx%d out of range [1, 16384]", c->width, c->height);
        return RGS_EINVAL;
    }
    if (!(c->near_z > 0) || !std::isfinite(c->near_z)) { set_error("camera: near_z must be > 0"); return RGS_EINVAL; }
    return RGS_OK;
}

int check_opts(const rgs_render_opts* o) {
    if (!o) { set_error("opts: NULL"); return RGS_EINVAL; }
    if (o->tile != kTile) { set_error("opts: tile must be %d", kTile); return RGS_EINVAL; }
    if (!(o->trunc_mult > 0) || !(o->alpha_min > 0) || !(o->alpha_max > o->alpha_min) || !(o->alpha_max < 1) ||
        !(o->eps_T >= 0) || !(o->dilation >= 0) || !std::isfinite(o->trunc_mult)) {
        set_error("opts: need trunc_mult > 0, 0 < alpha_min < alpha_max < 1, eps_T >= 0, dilation >= 0");
        return RGS_EINVAL;
    }
    if (o->cull_occluded != 0 && o->cull_occluded != 1) {
        set_error("opts: cull_occluded must be 0 or 1");
        return RGS_EINVAL;
    }
    if (o->group_binning < 0 || o->group_binning > 2) {
        set_error("opts: group_binning must be 0, 1 or 2");
        return RGS_EINVAL;
    }
    return RGS_OK;
}

void view_order_host(const rgs_kd* kd, const rgs_camera* cam, int32_t* order) {
    const int L = kd->b.L;
    double R[9], t[3], o[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) R[3 * r + c] = cam->viewmat[4 * r + c];
        t[r] = cam->viewmat[4 * r + 3];
    }
    for (int c = 0; c < 3; ++c) o[c] = -(R[c] * t[0] + R[3 + c] * t[1] + R[6 + c] * t[2]);
    // near-child-first traversal; the child holding o (o on the plane: left) goes first
    int n = 0;
    int stack[2 * kMaxKdDepth + 4];
    int sp = 0;
    stack[sp++] = 0;
    const int first_leaf = (1 << L) - 1;
    while (sp > 0) {
        int j = stack[--sp];
        if (j >= first_leaf) {
            order[n++] = j - first_leaf;
            continue;
        }
        double s = kd->b.split[j];
        bool left_first = o[kd->b.axis[j]] <= s;
        int nearc = left_first ? 2 * j + 1 : 2 * j + 2, farc = left_first ? 2 * j + 2 : 2 * j + 1;
        stack[sp++] = farc;
        stack[sp++] = nearc;
    }
}

void fill_view(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
               ViewParams* vp, TreeParams* tp) {
    memset(vp, 0, sizeof *vp);
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) vp->R[3 * r + c] = cam->viewmat[4 * r + c];
        vp->t[r] = cam->viewmat[4 * r + 3];
    }
    for (int c = 0; c < 3; ++c) {
        double oc = -((double)vp->R[c] * vp->t[0] + (double)vp->R[3 + c] * vp->t[1] + (double)vp->R[6 + c] * vp->t[2]);
        vp->o[c] = (float)oc;
    }
    vp->fx = cam->fx; vp->fy = cam->fy; vp->cx = cam->cx; vp->cy = cam->cy;
    vp->ifx = 1.f / cam->fx; vp->ify = 1.f / cam->fy;
    vp->near_z = cam->near_z;
    vp->W = cam->width; vp->H = cam->height;
    vp->tiles_x = (cam->width + kTile - 1) / kTile;
    vp->tiles_y = (cam->height + kTile - 1) / kTile;
    vp->trunc_mult = opts->trunc_mult; vp->eps_T = opts->eps_T;
    vp->alpha_min = opts->alpha_min; vp->alpha_max = opts->alpha_max; vp->dilation = opts->dilation;
    for (int c = 0; c < 3; ++c) vp->bg[c] = opts->bg[c];
    vp->cull_occluded = opts->cull_occluded;
    vp->L = kd->b.L;
    vp->K = 1 << kd->b.L;
    vp->bin_lo = 0;
    vp->bin_hi = vp->K;
    vp->sh_degree = g ? g->sh_degree : 0;
    int ntiles = vp->tiles_x * vp->tiles_y;
    int bits = 0;
    while ((1 << bits) < ntiles) ++bits;
    vp->tile_bits = bits;
    int32_t order[64];
    view_order_host(kd, cam, order);
    for (int r = 0; r < vp->K; ++r) {
        vp->order[r] = (int8_t)order[r];
        vp->rank_of[order[r]] = (int8_t)r;
    }
    memset(tp, 0, sizeof *tp);
    tp->L = kd->b.L;
    for (int j = 0; j < (1 << kd->b.L) - 1; ++j) {
        tp->axis[j] = kd->b.axis[j];
        tp->split[j] = kd->b.split[j];
    }
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

namespace {

// Carves the workspace; returns the bytes needed (b may be NULL to only measure).
size_t layout(char* base, int64_t N, int64_t tiles, int K, int64_t inst_cap, RasterBuffers* b, bool foot = false) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += a256(bytes);
        return p;
    };
    RasterBuffers t;
    memset(&t, 0, sizeof t);
    t.header = (unsigned long long*)take(256);
    t.rec = (float4*)take(sizeof(float4) * 3 * N);
    t.g2d = (float4*)take(sizeof(float4) * 3 * N);
    t.cnt = (uint32_t*)take(4 * N);
    t.rect = (ushort4*)take(8 * N);
    t.mask = (unsigned long long*)take(8 * N);
    t.dkey = (uint32_t*)take(4 * N);
    t.dkey_lo = (uint32_t*)take(4 * N);
    t.vis_pos = (uint32_t*)take(4 * N);
    t.skey = (uint32_t*)take(4 * N);
    t.sid = (uint32_t*)take(4 * N);
    t.skey_alt = (uint32_t*)take(4 * N);
    t.sid_alt = (uint32_t*)take(4 * N);
    t.ioff = (uint32_t*)take(4 * N);
    t.counters = (unsigned long long*)take(128);
    t.item_ctr = t.counters ? t.counters + 12 : nullptr;
    t.bin_ctr = t.counters ? t.counters + 14 : nullptr;
    // deferred emission: per launch a list of (id, base) for up to one splat in four (at
    // least 8192, at most 2^20)
    const int64_t ucap = N / 4 < 8192 ? 8192 : (N / 4 > (1 << 20) ? (1 << 20) : N / 4);
    t.units = (uint4*)take(sizeof(uint2) * 2 * (size_t)ucap);
    // items kept by the count: up to 8 per splat (at least 2^16, at most 2^27 records of 16 B)
    const int64_t icap = N * 8 < (1 << 16) ? (1 << 16) : (N * 8 > (1ll << 27) ? (1ll << 27) : N * 8);
    // binning in groups of ranks (image-only forward)
    t.cnt_bin = (uint32_t*)take(4 * (size_t)N);
    t.state = (float4*)take(sizeof(float4) * 256 * (size_t)tiles);
    t.open = (uint8_t*)take((size_t)tiles);
    t.open_prefix = (uint32_t*)take(4 * (2 * (size_t)tiles + 1));
    t.open_sat = (uint32_t*)take(4 * (2 * (size_t)tiles + 2));
    t.item_at = (uint32_t*)take(4 * (size_t)N);
    t.ibase = (uint32_t*)take(4 * (size_t)N);
    t.items = (uint4*)take(sizeof(uint4) * (size_t)icap);
    t.item_first_all = (uint32_t*)take(sizeof(uint32_t) * (size_t)icap);
    t.item_cap = (uint32_t)icap;
    t.unit_cap = (uint32_t)ucap;
    t.ranges = (uint2*)take(sizeof(uint2) * tiles * K);
    t.cull_chunk = (float2*)take(sizeof(float2) * (size_t)tiles * K / 16 + sizeof(float2) * 2048 * K);
    t.clip_plane = (float4*)take(sizeof(float4) * kClipTable);
    t.clip_margin = (float*)take(sizeof(float) * kClipTable);
    t.ikey = (uint32_t*)take(4 * inst_cap);
    t.ival = (uint32_t*)take(4 * inst_cap);
    t.ikey_alt = (uint32_t*)take(4 * inst_cap);
    t.ival_alt = (uint32_t*)take(4 * inst_cap);
    if (foot) {   // the foot reading's ball radii and its bound sort
        t.foot_side = (float4*)take(16 * N);
        t.fkey = (uint32_t*)take(4 * inst_cap);
        t.fidx = (uint32_t*)take(4 * inst_cap);
    }
    t.inst_cap = inst_cap;
    size_t tb = radix_temp_bytes(N > inst_cap ? N : inst_cap);
    size_t sb = scan_temp_bytes(N);
    t.temp_bytes = tb > sb ? tb : sb;
    t.temp = take(t.temp_bytes);
    if (b) *b = t;
    return off;
}

// The buffers of a workspace of ws_bytes, with the largest instance capacity that fits.
void carve_workspace(void* workspace, size_t ws_bytes, int64_t N, int64_t tiles, int K, RasterBuffers* b,
                     bool foot = false) {
    int64_t lo = 0, hi = (int64_t)(ws_bytes / 16) + 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (layout(nullptr, N, tiles, K, mid, nullptr, foot) <= ws_bytes) lo = mid; else hi = mid - 1;
    }
    layout((char*)workspace, N, tiles, K, lo, b, foot);
}

// ------------------------------------------------------------------ lists kept for the backward
// A forward with partial maps leaves in its workspace the records, the sorted instance
// payloads and the (tile, subset) ranges cut back to what it staged.  The backward of that
// same render replays exactly these lists, so when rgs_render_bwd gets the same workspace
// with the arguments of that forward it skips re-deriving them.  The host keeps, per
// workspace, the forward's arguments and a nonce that the forward also wrote into the
// workspace header; the backward takes the shortcut only when both match (anything that
// overwrote the header in between makes it re-derive the lists).
struct ListStamp {
    const rgs_kd* kd;
    rgs_gaussians g;
    rgs_camera cam;
    rgs_render_opts opts;
    const float* pC;
    const float* pT;
    const float* image;
    size_t ws_bytes;
    bool alt;           // payloads in ival_alt
    int64_t I;          // instances
    unsigned long long nonce;
};
std::mutex g_stamp_mu;
std::unordered_map<const void*, ListStamp> g_stamps;
std::atomic<unsigned long long> g_nonce_counter{0};

}  // namespace

unsigned long long next_nonce() {
    // splitmix64 of a per-process base and a counter: distinct per forward, never 0
    static const unsigned long long base = (unsigned long long)(uintptr_t)&g_nonce_counter ^
                                           ((unsigned long long)std::chrono::steady_clock::now().time_since_epoch().count()
                                            << 1);
    unsigned long long z = base + 0x9E3779B97F4A7C15ull * (g_nonce_counter.fetch_add(1) + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z ? z : 1;
}

namespace {

bool same_gaussians(const rgs_gaussians& a, const rgs_gaussians& b) {
    return a.means == b.means && a.log_scales == b.log_scales && a.quats == b.quats &&
           a.opacity_logits == b.opacity_logits && a.sh == b.sh && a.n == b.n && a.sh_degree == b.sh_degree;
}

void stamp_erase(const void* ws) {
    std::lock_guard<std::mutex> lk(g_stamp_mu);
    g_stamps.erase(ws);
}

struct PinnedCounters {
    unsigned long long* h = nullptr;
    ~PinnedCounters() {
        if (h) cudaFreeHost(h);
    }
};
thread_local PinnedCounters g_pinned;

// Projection, binning and sorting shared by the forward and the backward: on success
// `b` holds the records and the (tile, subset) ranges, and *sorted_ival the instance
// payloads in blend order.
// Binning in groups of ranks: build_lists bins the first group (view ranks [0, bin_hi))
// and leaves here what a later group needs.

struct GroupBins {
    bool grouped = false;                   // the render binned its first group only
    const uint32_t* sorted_ids = nullptr;   // the visible splats in depth order
    int64_t n_vis = 0;
    int64_t I0 = 0;                         // instances of the first group
    bool alt = false;                       // the sorted instances are in the alt buffers
};

int build_lists(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
                void* workspace, size_t ws_bytes, cudaStream_t s, ViewParams* vp, TreeParams* tp, RasterBuffers* b,
                const uint32_t** sorted_ival, const float* cull, unsigned long long* host_counters = nullptr,
                int64_t* n_inst = nullptr, bool foot = false, int bin_hi = -1, GroupBins* grp = nullptr,
                bool force_groups = false) {
    int rc;
    if ((rc = check_gaussians(g)) || (rc = check_camera(cam)) || (rc = check_opts(opts))) return rc;
    if (!kd) { set_error("render: NULL kd"); return RGS_EINVAL; }
    if (kd->b.L > kMaxRenderDepth) {
        set_error("render: KD depth %d > %d (at most 64 subsets per render)", kd->b.L, kMaxRenderDepth);
        return RGS_EINVAL;
    }
    fill_view(kd, g, cam, opts, vp, tp);
    vp->foot = foot ? 1 : 0;
    const int64_t N = g->n;
    const int64_t tiles = (int64_t)vp->tiles_x * vp->tiles_y;
    if (vp->tile_bits + vp->L > 32) { set_error("render: tile index and subset rank exceed 32 key bits"); return RGS_EINVAL; }
    size_t fixed = layout(nullptr, N, tiles, vp->K, 0, nullptr, foot);
    if (!workspace || ws_bytes < fixed) {
        set_required_workspace(layout(nullptr, N, tiles, vp->K, 1 << 20, nullptr, foot));
        set_error("render: workspace of %zu bytes is smaller than the %zu needed before binning", ws_bytes, fixed);
        return RGS_EOVERFLOW;
    }
    if (!aligned(workspace, 256)) { set_error("render: workspace must be 256-byte aligned"); return RGS_EINVAL; }
    carve_workspace(workspace, ws_bytes, N, tiles, vp->K, b, foot);
    b->cull = cull;
    // the projection counts the first group of ranks apart when the caller may bin in groups
    const bool two_counts = bin_hi > 0 && bin_hi < vp->K;
    if (two_counts) vp->bin_hi = bin_hi;
    else b->cnt_bin = nullptr;
    vp->set_clip(b->clip_plane, b->clip_margin);
    rc = launch_clip_table(*vp, *tp, s);
    if (rc) return rc;
    if (cull) {
        rc = launch_cull_chunks(*vp, cull, b->cull_chunk, s);
        if (rc) return rc;
    }

    RGS_CUDA_TRY(cudaMemsetAsync(b->counters, 0, 128, s));
    {
        ProfScope ps(ST_PROJECT, s);
        rc = launch_project_fwd(*g, *vp, *tp, *b, s);
    }
    if (rc) return rc;
    unsigned long long* hc = host_counters;
    if (!hc) {
        if (!g_pinned.h) RGS_CUDA_TRY(cudaMallocHost(&g_pinned.h, 64));
        hc = g_pinned.h;
    }
    RGS_CUDA_TRY(cudaMemcpyAsync(hc, b->counters, 16, cudaMemcpyDeviceToHost, s));
    unsigned long long first_group = 0;   // instances of the first group (pageable: a small copy)
    if (two_counts) RGS_CUDA_TRY(cudaMemcpyAsync(&first_group, b->counters + 14, 8, cudaMemcpyDeviceToHost, s));
    RGS_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t I_all = (int64_t)hc[0];
    const int64_t n_vis = (int64_t)hc[1];
    const bool grouped = two_counts && (force_groups || (I_all >= kGroupInstancesPerSplat * n_vis &&
                                                         I_all >= kGroupMinInstances));
    if (two_counts && !grouped) {   // one group after all: every rank, the items' full offsets
        vp->bin_hi = vp->K;
        b->item_first = b->item_first_all;
    }
    const int64_t I = grouped ? (int64_t)first_group : I_all;   // the instances binned now
    if (n_inst) *n_inst = I;
    if (I_all > 0xFFFFFFFFll - 1) {
        set_error("render: %lld tile instances exceed the 32-bit instance index", (long long)I_all);
        return RGS_EOVERFLOW;
    }
    if (I_all > b->inst_cap) {   // every group's instances fit in the count of all of them
        set_required_workspace(layout(nullptr, N, tiles, vp->K, I_all, nullptr, foot));
        set_error("render: %lld tile instances need a larger workspace", (long long)I_all);
        return RGS_EOVERFLOW;
    }
    prof_add_host_counts(I, n_vis);   // the instances binned (a later group adds its own)
    // compact the visible splats in index order, sort them by depth
    {
        ProfScope ps(ST_COMPACT, s);
        rc = exclusive_scan_u32(b->cnt, b->vis_pos, N, 1, nullptr, b->temp, b->temp_bytes, s);
        if (rc) return rc;
        compact_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(b->cnt, b->vis_pos, b->dkey_lo, N, b->skey,
                                                                   b->sid);
        RGS_CUDA_LAUNCH_CHECK();
    }
    // depth order as an LSD sort on (float bits of z, 16 bits below them): the low
    // digits first, then stably the float bits (sign bit 0: 31 bits)
    bool alt = false;
    const uint32_t* sorted_ids = nullptr;
    {
        ProfScope ps(ST_DEPTH_SORT, s);
        rc = radix_sort_pairs(b->skey, b->sid, b->skey_alt, b->sid_alt, n_vis, 16, b->temp, b->temp_bytes, s, &alt);
        if (rc) return rc;
        uint32_t* k1 = alt ? b->skey_alt : b->skey;
        uint32_t* v1 = alt ? b->sid_alt : b->sid;
        uint32_t* k2 = alt ? b->skey : b->skey_alt;
        uint32_t* v2 = alt ? b->sid : b->sid_alt;
        if (n_vis > 0) {
            gather_key_kernel<<<(unsigned)((n_vis + 255) / 256), 256, 0, s>>>(b->dkey, v1, n_vis, k1);
            RGS_CUDA_LAUNCH_CHECK();
        }
        bool alt2 = false;
        rc = radix_sort_pairs(k1, v1, k2, v2, n_vis, 31, b->temp, b->temp_bytes, s, &alt2);
        if (rc) return rc;
        sorted_ids = alt2 ? v2 : v1;
    }
    // instance offsets in depth order, emission, (tile, rank) sort, ranges
    {
        ProfScope ps(ST_OFFSETS, s);
        rc = exclusive_scan_u32(grouped ? b->cnt_bin : b->cnt, b->ioff, n_vis, 2, sorted_ids, b->temp, b->temp_bytes,
                                s);
        if (rc) return rc;
    }
    {
        ProfScope ps(ST_EMIT, s);
        rc = launch_emit(*vp, *tp, *b, sorted_ids, n_vis, s);
        if (rc) return rc;
    }
    const uint32_t* keys = nullptr;
    if (foot) {
        // per (tile, subset) run, ascending bound of the foot's ray parameter over the tile
        ProfScope ps(ST_INST_SORT, s);
        rc = launch_foot_order(*vp, *b, I, s, &keys, sorted_ival);
        if (rc) return rc;
    } else {
        {
            ProfScope ps(ST_INST_SORT, s);
            rc = radix_sort_pairs(b->ikey, b->ival, b->ikey_alt, b->ival_alt, I, vp->tile_bits + vp->L, b->temp,
                                  b->temp_bytes, s, &alt);
            if (rc) return rc;
        }
        keys = alt ? b->ikey_alt : b->ikey;
        *sorted_ival = alt ? b->ival_alt : b->ival;
    }
    if (grp) {
        grp->grouped = grouped;
        grp->sorted_ids = sorted_ids;
        grp->n_vis = n_vis;
        grp->I0 = I;
        grp->alt = alt;
    }
    ProfScope ps(ST_RANGES, s);
    rc = launch_ranges(keys, I, b->ranges, tiles * vp->K, s);
    return rc;
}

// The second group of a grouped image-only forward, after the first group's blend: view
// ranks [vp->bin_hi, K) in the tiles that blend left open.  Counts them per visible splat
// (in depth order), emits them after the first group's instances, sorts them (into the
// buffer that holds the first group's), adds their (tile, subset) ranges; returns their
// number in *I1 and in *any_open whether the first group left any tile open.
int bin_second_group(ViewParams* vp, const TreeParams& tp, const RasterBuffers& b, const GroupBins& grp,
                     int64_t* I1, bool* any_open, cudaStream_t s) {
    int rc;
    const int64_t tiles = (int64_t)vp->tiles_x * vp->tiles_y;
    vp->bin_lo = vp->bin_hi;
    vp->bin_hi = vp->K;
    vp->set_open(b.open_prefix, b.open_sat);
    unsigned long long n1 = 0;
    {
        ProfScope ps(ST_OFFSETS, s);
        if ((rc = launch_open_prefix(*vp, b.open, b.open_prefix, b.open_sat, s))) return rc;
        // no tile left open (the first group saturated every one): nothing more to bin
        uint32_t open_tiles = 0;
        const size_t last = (size_t)vp->tiles_y * ((size_t)vp->tiles_x + 1) + (size_t)vp->tiles_x;
        RGS_CUDA_TRY(cudaMemcpyAsync(&open_tiles, b.open_sat + last, 4, cudaMemcpyDeviceToHost, s));
        RGS_CUDA_TRY(cudaStreamSynchronize(s));
        *any_open = open_tiles != 0;
        if (open_tiles == 0) {
            *I1 = 0;
            return RGS_OK;
        }
        // work queues [4, 12) and the group's total [15]; [12] (the kept items) stays
        RGS_CUDA_TRY(cudaMemsetAsync(b.counters + 4, 0, 8 * 8, s));
        RGS_CUDA_TRY(cudaMemsetAsync(b.counters + 15, 0, 8, s));
        if ((rc = launch_recount(*vp, tp, b, grp.sorted_ids, grp.n_vis, b.vis_pos, s))) return rc;
        if ((rc = exclusive_scan_u32(b.vis_pos, b.ioff, grp.n_vis, 0, nullptr, b.temp, b.temp_bytes, s))) return rc;
        RGS_CUDA_TRY(cudaMemcpyAsync(&n1, b.counters + 15, 8, cudaMemcpyDeviceToHost, s));
        RGS_CUDA_TRY(cudaMemsetAsync(b.counters + 4, 0, 8, s));   // the emission's work queue
        RGS_CUDA_TRY(cudaStreamSynchronize(s));
    }
    *I1 = (int64_t)n1;
    prof_add_host_counts(*I1, 0);
    const int64_t I0 = grp.I0;
    if (I0 + *I1 > b.inst_cap) {   // cannot happen: both groups are counted in the total
        set_error("render: the second group's %lld instances overflow the workspace", (long long)*I1);
        return RGS_EOVERFLOW;
    }
    if (*I1 == 0) return RGS_OK;
    RasterBuffers b2 = b;
    b2.ikey = b.ikey + I0;
    b2.ival = b.ival + I0;
    {
        ProfScope ps(ST_EMIT, s);
        if ((rc = launch_emit(*vp, tp, b2, grp.sorted_ids, grp.n_vis, s))) return rc;
    }
    bool alt1 = false;
    {
        ProfScope ps(ST_INST_SORT, s);
        rc = radix_sort_pairs(b.ikey + I0, b.ival + I0, b.ikey_alt + I0, b.ival_alt + I0, *I1, vp->tile_bits + vp->L,
                              b.temp, b.temp_bytes, s, &alt1);
        if (rc) return rc;
        if (alt1 != grp.alt) {   // a pass count of other parity (a group of at most one instance)
            uint32_t* dk = grp.alt ? b.ikey_alt : b.ikey;
            uint32_t* dv = grp.alt ? b.ival_alt : b.ival;
            const uint32_t* sk = alt1 ? b.ikey_alt : b.ikey;
            const uint32_t* sv = alt1 ? b.ival_alt : b.ival;
            RGS_CUDA_TRY(cudaMemcpyAsync(dk + I0, sk + I0, 4 * (size_t)*I1, cudaMemcpyDeviceToDevice, s));
            RGS_CUDA_TRY(cudaMemcpyAsync(dv + I0, sv + I0, 4 * (size_t)*I1, cudaMemcpyDeviceToDevice, s));
        }
    }
    const uint32_t* keys = grp.alt ? b.ikey_alt : b.ikey;
    ProfScope ps(ST_RANGES, s);
    return launch_ranges(keys + I0, *I1, b.ranges, tiles * vp->K, s, (uint32_t)I0, false);
}

}  // namespace

int render_fwd_into(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
                    float* partial_C, float* partial_T, float* image, float* T_final, float* tile_depth,
                    void* workspace, size_t ws_bytes, cudaStream_t s, unsigned long long* host_counters,
                    bool keep_lists) {
    if ((!partial_C) != (!partial_T) || (!partial_C && !image)) {
        set_error("render_fwd: give both partial maps, or neither together with an image (forward only)");
        return RGS_EINVAL;
    }
    ViewParams vp;
    TreeParams tp;
    RasterBuffers b;
    const uint32_t* ival = nullptr;
    int64_t I = 0;
    if (keep_lists) stamp_erase(workspace);   // its lists are about to be replaced
    // an image-only forward bins its subsets in two groups of view ranks (group_binning)
    const int K = kd ? 1 << kd->b.L : 1;
    const bool grouped = opts && opts->group_binning >= 1 && !partial_C && image && K >= 4;
    const int r1 = grouped ? (K / 8 > 1 ? K / 8 : 1) : K;
    GroupBins grp;
    int rc = build_lists(kd, g, cam, opts, workspace, ws_bytes, s, &vp, &tp, &b, &ival, nullptr, host_counters, &I,
                         false, r1, grouped ? &grp : nullptr, opts && opts->group_binning == 2);
    if (rc) return rc;
    const bool keep = keep_lists && (partial_C != nullptr || image != nullptr);   // a backward may follow
    const bool two = grouped && grp.grouped;
    {
        ProfScope ps(ST_BLEND_FWD, s);
        rc = launch_blend_fwd(vp, tp, b, ival, partial_C, partial_T, image, T_final, tile_depth, s, keep, 0,
                              two ? r1 : K);
        if (rc) return rc;
    }
    if (two) {
        int64_t I1 = 0;
        bool any_open = false;
        if ((rc = bin_second_group(&vp, tp, b, grp, &I1, &any_open, s))) return rc;
        if (any_open) {   // (every closed tile has its image already)
            ProfScope ps(ST_BLEND_FWD, s);
            rc = launch_blend_fwd(vp, tp, b, ival, nullptr, nullptr, image, T_final, tile_depth, s, keep, r1, K);
            if (rc) return rc;
        }
        I += I1;
    }
    if (keep) {
        ListStamp st;
        st.kd = kd;
        st.g = *g;
        st.cam = *cam;
        st.opts = *opts;
        st.pC = partial_C;
        st.pT = partial_T;
        st.image = image;
        st.ws_bytes = ws_bytes;
        st.alt = ival == b.ival_alt;
        st.I = I;
        st.nonce = next_nonce();
        store_u64_kernel<<<1, 1, 0, s>>>(b.header, st.nonce);
        RGS_CUDA_LAUNCH_CHECK();
        std::lock_guard<std::mutex> lk(g_stamp_mu);
        g_stamps[workspace] = st;
    }
    return RGS_OK;
}

// The backward of the forward whose lists `workspace` holds, if the arguments are that
// forward's: replays its lists (no projection, sorting or emission).  Returns 1 when it
// does not apply (the caller re-derives the lists), else a status.  image != nullptr: the
// flat form (the forward's image must be the one given; its partial maps are not read).
int render_bwd_reuse(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
                     const float* partial_C, const float* partial_T, const float* image, const float* dL_dimage,
                     const rgs_gaussian_grads* grads, void* workspace, size_t ws_bytes, cudaStream_t s) {
    ListStamp st;
    {
        std::lock_guard<std::mutex> lk(g_stamp_mu);
        auto it = g_stamps.find(workspace);
        if (it == g_stamps.end()) return 1;
        st = it->second;
    }
    const bool same_maps = image ? st.image == image : (st.pC == partial_C && st.pT == partial_T);
    if (st.kd != kd || !same_gaussians(st.g, *g) || memcmp(&st.cam, cam, sizeof *cam) != 0 ||
        memcmp(&st.opts, opts, sizeof *opts) != 0 || !same_maps || st.ws_bytes != ws_bytes)
        return 1;
    ViewParams vp;
    TreeParams tp;
    fill_view(kd, g, cam, opts, &vp, &tp);
    RasterBuffers b;
    carve_workspace(workspace, ws_bytes, g->n, (int64_t)vp.tiles_x * vp.tiles_y, vp.K, &b);
    vp.set_clip(b.clip_plane, b.clip_margin);   // the forward's table, still in the workspace
    if (st.I > b.inst_cap) return 1;
    unsigned long long* hc = g_pinned.h;
    if (!hc) {
        RGS_CUDA_TRY(cudaMallocHost(&g_pinned.h, 64));
        hc = g_pinned.h;
    }
    RGS_CUDA_TRY(cudaMemcpyAsync(hc, b.header, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    RGS_CUDA_TRY(cudaStreamSynchronize(s));
    if (hc[0] != st.nonce) return 1;   // the workspace was overwritten since
    const uint32_t* ival = st.alt ? b.ival_alt : b.ival;
    int rc;
    {
        ProfScope ps(ST_BLEND_BWD, s);
        RGS_CUDA_TRY(cudaMemsetAsync(b.g2d, 0, sizeof(float4) * 3 * (size_t)g->n, s));
        rc = launch_blend_bwd(vp, tp, b, ival, partial_C, partial_T, image, dL_dimage, st.I, g->n, s);
        if (rc) return rc;
    }
    ProfScope ps(ST_PROJECT_BWD, s);
    return launch_project_bwd(*g, *grads, vp, b, s);
}

// Both backward forms: replay the forward's lists if the workspace holds them, else
// re-derive them (depth-culled by tile_depth when given).
int render_bwd_any(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
                   const float* partial_C, const float* partial_T, const float* image, const float* dL_dimage,
                   const float* tile_depth, const rgs_gaussian_grads* grads, void* workspace, size_t ws_bytes,
                   cudaStream_t s) {
    if (!dL_dimage || !grads || !grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits ||
        !grads->sh) {
        set_error("render_bwd: NULL argument");
        return RGS_EINVAL;
    }
    if (!aligned(grads->quats, 16)) { set_error("render_bwd: grads->quats must be 16-byte aligned"); return RGS_EINVAL; }
    int rc;
    if ((rc = check_gaussians(g)) || (rc = check_camera(cam)) || (rc = check_opts(opts))) return rc;
    if (!kd) { set_error("render: NULL kd"); return RGS_EINVAL; }
    rc = render_bwd_reuse(kd, g, cam, opts, partial_C, partial_T, image, dL_dimage, grads, workspace, ws_bytes, s);
    if (rc != 1) return rc;
    // re-derive the lists (depth-culled by tile_depth when given)
    stamp_erase(workspace);
    ViewParams vp;
    TreeParams tp;
    RasterBuffers b;
    const uint32_t* ival = nullptr;
    int64_t I = 0;
    rc = build_lists(kd, g, cam, opts, workspace, ws_bytes, s, &vp, &tp, &b, &ival, tile_depth, nullptr, &I);
    if (rc) return rc;
    {
        ProfScope ps(ST_BLEND_BWD, s);
        RGS_CUDA_TRY(cudaMemsetAsync(b.g2d, 0, sizeof(float4) * 3 * (size_t)g->n, s));
        rc = launch_blend_bwd(vp, tp, b, ival, partial_C, partial_T, image, dL_dimage, I, g->n, s);
        if (rc) return rc;
    }
    ProfScope ps(ST_PROJECT_BWD, s);
    return launch_project_bwd(*g, *grads, vp, b, s);
}

}  // namespace rgs

using namespace rgs;

extern "C" {

const char* rgs_last_error(void) { return g_err; }
size_t rgs_last_required_workspace(void) { return g_required; }
int rgs_version(void) { return 100; }

void rgs_default_opts(rgs_render_opts* o) {
    if (!o) return;
    o->tile = kTile;
    o->trunc_mult = 3.f;
    o->eps_T = 1e-6f;
    o->alpha_min = 1.f / 255.f;
    o->alpha_max = 0.99f;
    o->dilation = 0.3f;
    o->bg[0] = o->bg[1] = o->bg[2] = 0.f;
    o->cull_occluded = 0;
    o->group_binning = 1;
}

int rgs_kd_partition(const rgs_gaussians* g, int depth_L, float trunc_mult, rgs_kd** out, void* stream) {
    if (!out) { set_error("kd_partition: out is NULL"); return RGS_EINVAL; }
    *out = nullptr;
    if (!g || !g->means || !g->log_scales || g->n < 1 || g->n > 0x7fffffffll) {
        set_error("kd_partition: need means, log_scales and 1 <= n < 2^31");
        return RGS_EINVAL;
    }
    if (depth_L < 0 || depth_L > kMaxKdDepth) { set_error("kd_partition: depth %d not in [0, %d]", depth_L, kMaxKdDepth); return RGS_EINVAL; }
    if (!(trunc_mult > 0) || !std::isfinite(trunc_mult)) { set_error("kd_partition: trunc_mult must be > 0"); return RGS_EINVAL; }
    rgs_kd* kd = new (std::nothrow) rgs_kd;
    if (!kd) { set_error("kd_partition: out of host memory"); return RGS_ENOMEM; }
    cudaGetDevice(&kd->device);
    kd->trunc_mult = trunc_mult;
    int rc;
    {
        ProfScope ps(ST_KD, (cudaStream_t)stream);
        rc = kd_build(*g, depth_L, trunc_mult, &kd->b, (cudaStream_t)stream);
    }
    if (rc != RGS_OK) {
        if (kd->b.idx_dev) cudaFree(kd->b.idx_dev);
        delete kd;
        return rc;
    }
    *out = kd;
    return RGS_OK;
}

int rgs_kd_from_splits(const rgs_gaussians* g, int depth_L, const int32_t* axis_host, const float* split_host,
                       float trunc_mult, rgs_kd** out, void* stream) {
    if (!out) { set_error("kd_from_splits: out is NULL"); return RGS_EINVAL; }
    *out = nullptr;
    if (!g || !g->means || !g->log_scales || g->n < 1 || g->n > 0x7fffffffll) {
        set_error("kd_from_splits: need means, log_scales and 1 <= n < 2^31");
        return RGS_EINVAL;
    }
    if (depth_L < 0 || depth_L > kMaxKdDepth) { set_error("kd_from_splits: depth %d not in [0, %d]", depth_L, kMaxKdDepth); return RGS_EINVAL; }
    if (!(trunc_mult > 0) || !std::isfinite(trunc_mult)) { set_error("kd_from_splits: trunc_mult must be > 0"); return RGS_EINVAL; }
    const int nn = (1 << depth_L) - 1;
    if (nn > 0 && (!axis_host || !split_host)) { set_error("kd_from_splits: NULL splits"); return RGS_EINVAL; }
    for (int j = 0; j < nn; ++j) {
        if (axis_host[j] < 0 || axis_host[j] > 2 || !std::isfinite(split_host[j])) {
            set_error("kd_from_splits: node %d has axis %d / split %g", j, axis_host[j], (double)split_host[j]);
            return RGS_EINVAL;
        }
    }
    rgs_kd* kd = new (std::nothrow) rgs_kd;
    if (!kd) { set_error("kd_from_splits: out of host memory"); return RGS_ENOMEM; }
    cudaGetDevice(&kd->device);
    kd->trunc_mult = trunc_mult;
    memset(&kd->b, 0, sizeof kd->b);
    kd->b.L = depth_L;
    for (int j = 0; j < nn; ++j) {
        kd->b.axis[j] = (int8_t)axis_host[j];
        kd->b.split[j] = split_host[j];
    }
    int rc;
    {
        ProfScope ps(ST_KD, (cudaStream_t)stream);
        rc = kd_subsets(*g, trunc_mult, &kd->b, (cudaStream_t)stream);
    }
    if (rc != RGS_OK) {
        if (kd->b.idx_dev) cudaFree(kd->b.idx_dev);
        delete kd;
        return rc;
    }
    *out = kd;
    return RGS_OK;
}

int rgs_kd_info(const rgs_kd* kd, int* depth_L, int* K, int64_t* total) {
    if (!kd) { set_error("kd_info: NULL"); return RGS_EINVAL; }
    if (depth_L) *depth_L = kd->b.L;
    if (K) *K = 1 << kd->b.L;
    if (total) *total = kd->b.M;
    return RGS_OK;
}

int rgs_kd_splits(const rgs_kd* kd, int32_t* axis_host, float* split_host) {
    if (!kd) { set_error("kd_splits: NULL"); return RGS_EINVAL; }
    int nn = (1 << kd->b.L) - 1;
    for (int j = 0; j < nn; ++j) {
        if (axis_host) axis_host[j] = kd->b.axis[j];
        if (split_host) split_host[j] = kd->b.split[j];
    }
    return RGS_OK;
}

int rgs_kd_subsets(const rgs_kd* kd, int64_t* offsets_host, int32_t* idx_dev) {
    if (!kd || !offsets_host) { set_error("kd_subsets: NULL argument"); return RGS_EINVAL; }
    int K = 1 << kd->b.L;
    for (int k = 0; k <= K; ++k) offsets_host[k] = kd->b.offsets[k];
    if (idx_dev) RGS_CUDA_TRY(cudaMemcpy(idx_dev, kd->b.idx_dev, sizeof(int32_t) * kd->b.M, cudaMemcpyDeviceToDevice));
    return RGS_OK;
}

int rgs_kd_destroy(rgs_kd* kd) {
    if (!kd) return RGS_OK;
    if (kd->b.idx_dev) cudaFree(kd->b.idx_dev);
    delete kd;
    return RGS_OK;
}

int rgs_view_order(const rgs_kd* kd, const rgs_camera* cam, int32_t* order_host) {
    if (!kd || !order_host) { set_error("view_order: NULL argument"); return RGS_EINVAL; }
    int rc = check_camera(cam);
    if (rc) return rc;
    view_order_host(kd, cam, order_host);
    return RGS_OK;
}

int rgs_render_workspace_size(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam,
                              const rgs_render_opts* opts, int64_t instance_capacity, size_t* bytes) {
    int rc;
    if (!kd || !bytes) { set_error("workspace_size: NULL argument"); return RGS_EINVAL; }
    if ((rc = check_gaussians(g)) || (rc = check_camera(cam)) || (rc = check_opts(opts))) return rc;
    if (instance_capacity < 0) { set_error("workspace_size: negative capacity"); return RGS_EINVAL; }
    int64_t tiles = (int64_t)((cam->width + kTile - 1) / kTile) * ((cam->height + kTile - 1) / kTile);
    *bytes = layout(nullptr, g->n, tiles, 1 << kd->b.L, instance_capacity, nullptr);
    return RGS_OK;
}

int rgs_render_fwd(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
                   float* partial_C, float* partial_T, float* image, float* T_final, float* tile_depth,
                   void* workspace, size_t ws_bytes, void* stream) {
    return render_fwd_into(kd, g, cam, opts, partial_C, partial_T, image, T_final, tile_depth, workspace, ws_bytes,
                           (cudaStream_t)stream, nullptr);
}

int rgs_render_fwd_foot(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam,
                        const rgs_render_opts* opts, float* partial_C, float* partial_T, float* image,
                        float* T_final, void* workspace, size_t ws_bytes, uint64_t* overflow_host, void* stream) {
    if ((!partial_C) != (!partial_T) || (!partial_C && !image)) {
        set_error("render_fwd_foot: give both partial maps, or neither together with an image");
        return RGS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    stamp_erase(workspace);   // its lists are about to be replaced
    ViewParams vp;
    TreeParams tp;
    RasterBuffers b;
    const uint32_t* ival = nullptr;
    int64_t I = 0;
    int rc = build_lists(kd, g, cam, opts, workspace, ws_bytes, s, &vp, &tp, &b, &ival, nullptr, nullptr, &I, true);
    if (rc) return rc;
    // the overflow counter: word 6 of the workspace counter block (unused by the lists)
    unsigned long long* over = b.counters + 6;
    RGS_CUDA_TRY(cudaMemsetAsync(over, 0, 8, s));
    {
        ProfScope ps(ST_BLEND_FWD, s);
        rc = launch_blend_foot(vp, tp, b, ival, partial_C, partial_T, image, T_final, over, s);
        if (rc) return rc;
    }
    if (overflow_host) {
        if (!g_pinned.h) RGS_CUDA_TRY(cudaMallocHost(&g_pinned.h, 64));
        unsigned long long* h = g_pinned.h;
        RGS_CUDA_TRY(cudaMemcpyAsync(h + 6, over, 8, cudaMemcpyDeviceToHost, s));
        RGS_CUDA_TRY(cudaStreamSynchronize(s));
        *overflow_host = (uint64_t)h[6];
    }
    return RGS_OK;
}

int rgs_render_bwd_foot(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam,
                        const rgs_render_opts* opts, const float* image, const float* dL_dimage,
                        const rgs_gaussian_grads* grads, void* workspace, size_t ws_bytes, uint64_t* overflow_host,
                        void* stream) {
    if (!image || !dL_dimage || !grads || !grads->means || !grads->log_scales || !grads->quats ||
        !grads->opacity_logits || !grads->sh) {
        set_error("render_bwd_foot: NULL argument");
        return RGS_EINVAL;
    }
    if (!aligned(grads->quats, 16)) {
        set_error("render_bwd_foot: grads->quats must be 16-byte aligned");
        return RGS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    stamp_erase(workspace);   // its lists are about to be replaced
    ViewParams vp;
    TreeParams tp;
    RasterBuffers b;
    const uint32_t* ival = nullptr;
    int64_t I = 0;
    int rc = build_lists(kd, g, cam, opts, workspace, ws_bytes, s, &vp, &tp, &b, &ival, nullptr, nullptr, &I, true);
    if (rc) return rc;
    unsigned long long* over = b.counters + 6;
    RGS_CUDA_TRY(cudaMemsetAsync(over, 0, 8, s));
    {
        ProfScope ps(ST_BLEND_BWD, s);
        RGS_CUDA_TRY(cudaMemsetAsync(b.g2d, 0, sizeof(float4) * 3 * (size_t)g->n, s));
        rc = launch_blend_foot_bwd(vp, tp, b, ival, image, dL_dimage, over, s);
        if (rc) return rc;
    }
    {
        ProfScope ps(ST_PROJECT_BWD, s);
        rc = launch_project_bwd(*g, *grads, vp, b, s);
        if (rc) return rc;
    }
    if (overflow_host) {
        if (!g_pinned.h) RGS_CUDA_TRY(cudaMallocHost(&g_pinned.h, 64));
        unsigned long long* h = g_pinned.h;
        RGS_CUDA_TRY(cudaMemcpyAsync(h + 6, over, 8, cudaMemcpyDeviceToHost, s));
        RGS_CUDA_TRY(cudaStreamSynchronize(s));
        *overflow_host = (uint64_t)h[6];
    }
    return RGS_OK;
}

int rgs_render_bwd(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
                   const float* partial_C, const float* partial_T, const float* dL_dimage, const float* tile_depth,
                   const rgs_gaussian_grads* grads, void* workspace, size_t ws_bytes, void* stream) {
    if (!partial_C || !partial_T) {
        set_error("render_bwd: NULL partial maps");
        return RGS_EINVAL;
    }
    return render_bwd_any(kd, g, cam, opts, partial_C, partial_T, nullptr, dL_dimage, tile_depth, grads, workspace,
                          ws_bytes, (cudaStream_t)stream);
}

int rgs_render_bwd_flat(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam, const rgs_render_opts* opts,
                        const float* image, const float* dL_dimage, const float* tile_depth,
                        const rgs_gaussian_grads* grads, void* workspace, size_t ws_bytes, void* stream) {
    if (!image) {
        set_error("render_bwd_flat: NULL image");
        return RGS_EINVAL;
    }
    return render_bwd_any(kd, g, cam, opts, nullptr, nullptr, image, dL_dimage, tile_depth, grads, workspace, ws_bytes,
                          (cudaStream_t)stream);
}

int rgs_merge_partials(const float* partial_C, const float* partial_T, const int32_t* order_dev, int K, int H, int W,
                       const float bg[3], float* image, float* T_out, void* stream) {
    if (!partial_C || !partial_T || !order_dev || !image || !bg || K < 1 || H < 1 || W < 1) {
        set_error("merge_partials: invalid argument");
        return RGS_EINVAL;
    }
    ProfScope ps(ST_MERGE, (cudaStream_t)stream);
    return launch_merge(partial_C, partial_T, order_dev, K, H, W, bg, image, T_out, (cudaStream_t)stream);
}

int rgs_merge_partials_bwd(const float* partial_C, const float* partial_T, const int32_t* order_dev, int K, int H,
                           int W, const float bg[3], const float* dL_dimage, const float* dL_dT_out,
                           float* dL_dpartial_C, float* dL_dpartial_T, void* stream) {
    if (!partial_C || !partial_T || !order_dev || !bg || !dL_dimage || !dL_dpartial_C || !dL_dpartial_T || K < 1 ||
        H < 1 || W < 1) {
        set_error("merge_partials_bwd: invalid argument");
        return RGS_EINVAL;
    }
    ProfScope ps(ST_MERGE_BWD, (cudaStream_t)stream);
    return launch_merge_bwd(partial_C, partial_T, order_dev, K, H, W, bg, dL_dimage, dL_dT_out, dL_dpartial_C,
                            dL_dpartial_T, (cudaStream_t)stream);
}

size_t rgs_sort_temp_bytes(int64_t n) { return radix_temp_bytes(n > 0 ? n : 1); }

int rgs_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, int64_t n, int end_bit,
                   void* temp, size_t temp_bytes, void* stream, int* in_alt) {
    if (!in_alt || n < 0 || end_bit < 1 || end_bit > 32) {
        set_error("sort_pairs: invalid argument");
        return RGS_EINVAL;
    }
    *in_alt = 0;
    if (n == 0) return RGS_OK;
    if (!keys || !vals || !keys_alt || !vals_alt || !temp) {
        set_error("sort_pairs: NULL array");
        return RGS_EINVAL;
    }
    bool alt = false;
    const int rc = radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, end_bit, temp, temp_bytes, (cudaStream_t)stream,
                                    &alt);
    *in_alt = alt ? 1 : 0;
    return rc;
}

int rgs_adam_step(float* param, float* grad, float* m, float* v, int64_t n, const int64_t* seg_offsets_host,
                  const float* seg_lr_host, int nseg, float beta1, float beta2, float eps, int step, int zero_grad,
                  void* stream) {
    return rgs_adam_step_periodic(param, grad, m, v, n, seg_offsets_host, seg_lr_host, nseg, -1, 1, 0, 0.f, beta1,
                                  beta2, eps, step, zero_grad, stream);
}

int rgs_adam_step_periodic(float* param, float* grad, float* m, float* v, int64_t n, const int64_t* seg_offsets_host,
                           const float* seg_lr_host, int nseg, int pseg, int64_t period, int64_t head, float head_lr,
                           float beta1, float beta2, float eps, int step, int zero_grad, void* stream) {
    if (!param || !grad || !m || !v || n < 1 || !seg_offsets_host || !seg_lr_host || nseg < 1 || nseg > 16 || step < 1) {
        set_error("adam_step: invalid argument");
        return RGS_EINVAL;
    }
    if (pseg >= nseg || (pseg >= 0 && (period < 1 || head < 0 || head > period))) {
        set_error("adam_step: periodic rule needs 0 <= pseg < nseg, period >= 1, 0 <= head <= period");
        return RGS_EINVAL;
    }
    if (!aligned(param, 16) || !aligned(grad, 16) || !aligned(m, 16) || !aligned(v, 16)) {
        set_error("adam_step: buffers must be 16-byte aligned");
        return RGS_EINVAL;
    }
    if (seg_offsets_host[0] != 0 || seg_offsets_host[nseg] != n) {
        set_error("adam_step: segments must cover [0, n)");
        return RGS_EINVAL;
    }
    float bc1 = (float)(1.0 / (1.0 - std::pow((double)beta1, step)));
    float bc2 = (float)(1.0 / (1.0 - std::pow((double)beta2, step)));
    ProfScope ps(ST_ADAM, (cudaStream_t)stream);
    return launch_adam(param, grad, m, v, n, seg_offsets_host, seg_lr_host, nseg, beta1, beta2, eps, bc1, bc2,
                       zero_grad, (cudaStream_t)stream, pseg < 0 ? -1 : pseg, pseg < 0 ? 1 : period, head, head_lr);
}

int rgs_profile_enable(int flags) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if ((flags & 2) && !g_prof.dev_pairs) {
        RGS_CUDA_TRY(cudaMalloc(&g_prof.dev_pairs, 16 * sizeof(unsigned long long)));
        RGS_CUDA_TRY(cudaMemset(g_prof.dev_pairs, 0, 16 * sizeof(unsigned long long)));
    }
    g_prof.on = (flags & 1) != 0;
    g_prof.count = (flags & 2) != 0;
    return RGS_OK;
}

int rgs_profile_num_stages(void) { return ST_COUNT; }

const char* rgs_profile_stage_name(int stage) { return (stage >= 0 && stage < ST_COUNT) ? kStageNames[stage] : ""; }

int rgs_profile_read(double* ms_host, int64_t* launches_host, int64_t* counters_host, int reset) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (auto& r : g_prof.done) {
        RGS_CUDA_TRY(cudaEventSynchronize(r.b));
        float ms = 0.f;
        RGS_CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
        g_prof.ms[r.stage] += ms;
        g_prof.launches[r.stage] += 1;
        g_prof.pool.push_back(r.a);
        g_prof.pool.push_back(r.b);
    }
    g_prof.done.clear();
    for (int i = 0; i < ST_COUNT; ++i) {
        if (ms_host) ms_host[i] = g_prof.ms[i];
        if (launches_host) launches_host[i] = g_prof.launches[i];
    }
    unsigned long long pairs[16] = {};
    if (g_prof.dev_pairs) RGS_CUDA_TRY(cudaMemcpy(pairs, g_prof.dev_pairs, sizeof pairs, cudaMemcpyDeviceToHost));
    if (counters_host) {
        for (int i = 0; i < 4; ++i) counters_host[i] = (int64_t)pairs[i];
        counters_host[4] = g_prof.host_counts[0];
        counters_host[5] = g_prof.host_counts[1];
        counters_host[6] = g_launches.load();
        for (int i = 0; i < 9; ++i) counters_host[7 + i] = (int64_t)pairs[4 + i];
    }
    if (reset) {
        for (int i = 0; i < ST_COUNT; ++i) {
            g_prof.ms[i] = 0;
            g_prof.launches[i] = 0;
        }
        g_prof.host_counts[0] = g_prof.host_counts[1] = 0;
        g_launches.store(0);
        if (g_prof.dev_pairs) RGS_CUDA_TRY(cudaMemset(g_prof.dev_pairs, 0, 16 * sizeof(unsigned long long)));
    }
    return RGS_OK;
}

float rgs_position_lr(int64_t step, int64_t max_steps, float lr_init, float lr_final) {
    double t = max_steps > 0 ? (double)step / (double)max_steps : 1.0;
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    return (float)std::exp(std::log((double)lr_init) * (1.0 - t) + std::log((double)lr_final) * t);
}

}  // extern "C"
