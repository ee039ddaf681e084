// Render server: a resident scene, a host queue of forward-only render requests, and a
// scheduler thread that packs queued requests into batches and launches each batch as one
// captured CUDA graph (see the serving section of rgs.h).
//
// Batch pipeline (all counts stay on the device, so one graph per lane serves every
// batch whatever its views, resolutions and splat counts):
//   slot table H2D -> clear counters and tile ranges -> projection of every (request,
//   splat) pair -> compaction of the visible pairs -> depth sort (16 low bits, float bits
//   of z, then request: stable LSD, so the order is (request, depth, index)) -> instance
//   offsets -> capacity check -> emission with global tile keys -> instance sort ->
//   tile ranges -> persistent blend over (request, tile) work items -> counters D2H.
// Each request's arithmetic is that of rgs_render_fwd; a request's records, keys and
// tiles never mix with another's, so its image is the same alone and in any batch.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "rgs_internal.cuh"

namespace rgs {

namespace {

static_assert(sizeof(ViewParams) % 4 == 0, "view parameters are copied as 32-bit words");

// ------------------------------------------------------------------ batch kernels
inline unsigned grid_stride_blocks() { return (unsigned)sm_count() * 8; }   // the grid-stride passes

__device__ __forceinline__ int64_t dev_count(const unsigned long long* n, int64_t cap) {
    const unsigned long long v = *n;
    return v < (unsigned long long)cap ? (int64_t)v : cap;
}

// Visible (request, splat) pairs in index order: (16 low depth bits, pair id).
__global__ void compact_batch_kernel(const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ pos,
                                     const uint32_t* __restrict__ dkey_lo, const unsigned long long* __restrict__ n_dev,
                                     int64_t cap, uint32_t* __restrict__ skey, uint32_t* __restrict__ sid) {
    const int64_t n = dev_count(n_dev, cap);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        if (cnt[j] == 0) continue;
        const uint32_t p = pos[j];
        skey[p] = dkey_lo[j];
        sid[p] = (uint32_t)j;
    }
}

// key[p] = src[id[p]] (src = float bits of z), or id[p] / N (the request) when src is null.
__global__ void batch_key_kernel(const uint32_t* __restrict__ src, const uint32_t* __restrict__ id, int64_t N,
                                 const unsigned long long* __restrict__ n_dev, int64_t cap, uint32_t* __restrict__ key) {
    const int64_t n = dev_count(n_dev, cap);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        key[p] = src ? src[id[p]] : (uint32_t)(id[p] / (uint64_t)N);
}

// Overflow check: instances beyond the lane's capacity discard the batch.  grouped: the
// first binning group's instances are the ones sorted now (the total bounds every group's).
__global__ void check_capacity_kernel(unsigned long long* counters, int64_t inst_cap, bool grouped) {
    const unsigned long long I = counters[0];
    const bool over = I > (unsigned long long)inst_cap;
    counters[2] = over ? 1ull : 0ull;
    counters[4] = over ? 0ull : grouped ? counters[kBatchBinCounter] : I;
}

// The second binning group's instances go after the first group's.  The two groups' counts
// add up to at most the total by construction; a batch where they do not is failed
// (overflow flag 2) before anything is written past the first group.
__global__ void check_group2_kernel(unsigned long long* counters, int64_t inst_cap) {
    unsigned long long& n1 = counters[kBatchBinCounter + 1];
    if (counters[2]) {
        n1 = 0ull;
    } else if (counters[4] + n1 > (unsigned long long)inst_cap) {
        counters[2] = 2ull;
        n1 = 0ull;
    }
}

}  // namespace

// ------------------------------------------------------------------ lanes
// Carves one lane's buffers from `base` (NULL: measure); returns the bytes used.  train:
// also the per-(slot, splat) 2D-gradient records of a batched backward.
size_t lane_layout(char* base, int64_t N, int slots, int64_t tiles_cap, int K, int64_t inst_cap, LaneBufs* out,
                   bool train, int64_t group_tiles) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += a256(bytes);
        return p;
    };
    LaneBufs l;
    memset(&l, 0, sizeof l);
    const int64_t P = N * slots;   // (request, splat) pairs
    if (train) l.header = (unsigned long long*)take(256);
    l.slots = (BatchSlot*)take(sizeof(BatchSlot) * kMaxSlots);
    l.hdr = (BatchHeader*)take(sizeof(BatchHeader));
    l.counters = (unsigned long long*)take(8 * kBatchCounters);
    l.clip_plane = (float4*)take(sizeof(float4) * kMaxSlots * kClipTable);
    l.clip_margin = (float*)take(sizeof(float) * kMaxSlots * kClipTable);
    RasterBuffers& b = l.b;
    b.rec = (float4*)take(sizeof(float4) * 3 * P);
    b.cnt = (uint32_t*)take(4 * P);
    b.rect = (ushort4*)take(8 * P);
    b.mask = (unsigned long long*)take(8 * P);
    b.dkey = (uint32_t*)take(4 * P);
    b.dkey_lo = (uint32_t*)take(4 * P);
    b.vis_pos = (uint32_t*)take(4 * P);
    b.skey = (uint32_t*)take(4 * P);
    b.sid = (uint32_t*)take(4 * P);
    b.skey_alt = (uint32_t*)take(4 * P);
    b.sid_alt = (uint32_t*)take(4 * P);
    b.ioff = (uint32_t*)take(4 * P);
    // items the projection keeps for the emission: up to 4 per (request, splat) pair, at
    // most 2^26 records
    const int64_t icap = P * 4 < (1 << 16) ? (1 << 16) : (P * 4 > (1ll << 26) ? (1ll << 26) : P * 4);
    b.item_at = (uint32_t*)take(4 * P);
    b.ibase = (uint32_t*)take(4 * P);
    b.items = (uint4*)take(sizeof(uint4) * (size_t)icap);
    b.item_cap = (uint32_t)icap;
    b.item_ctr = l.counters ? l.counters + kBatchItemCounter : nullptr;
    if (train) b.g2d = (float4*)take(sizeof(float4) * 3 * P);
    if (group_tiles > 0) {
        // the group state of up to group_tiles tiles of the batch's grouped requests; per
        // slot, its tables take tiles_y (tiles_x + 1) <= 2 tiles prefix entries and
        // (tiles_y + 1)(tiles_x + 1) <= 3 tiles + 1 summed-area entries
        b.cnt_bin = (uint32_t*)take(4 * P);
        b.bin_ctr = l.counters ? l.counters + kBatchBinCounter : nullptr;
        l.group_tiles = group_tiles;
        b.state = (float4*)take(sizeof(float4) * (size_t)kTilePixels * (size_t)group_tiles);
        b.open = (uint8_t*)take((size_t)tiles_cap);
        l.prefix_cap = 2 * tiles_cap + slots;
        l.sat_cap = 3 * tiles_cap + 2 * slots;
        b.open_prefix = (uint32_t*)take(4 * (size_t)l.prefix_cap);
        b.open_sat = (uint32_t*)take(4 * (size_t)l.sat_cap);
        l.slots2 = (BatchSlot*)take(sizeof(BatchSlot) * kMaxSlots);
    }
    l.one = (unsigned long long*)take(8);
    b.ranges = (uint2*)take(sizeof(uint2) * tiles_cap * K);
    b.ikey = (uint32_t*)take(4 * inst_cap);
    b.ival = (uint32_t*)take(4 * inst_cap);
    b.ikey_alt = (uint32_t*)take(4 * inst_cap);
    b.ival_alt = (uint32_t*)take(4 * inst_cap);
    b.inst_cap = inst_cap;
    const size_t tr = radix_dev_temp_bytes(), ts = scan_dev_temp_bytes();
    b.temp_bytes = tr > ts ? tr : ts;
    b.temp = take(b.temp_bytes);
    if (out) *out = l;
    return off;
}

// A per-request blend launch during the capture of a lane's graph, with arguments that do
// nothing (each batch sets its own before the graph runs), and its graph node.
int capture_blend_node(const LaneBufs& l, const TreeParams& tp, cudaStream_t s, cudaGraphNode_t* node) {
    BlendNodeArgs a;
    memset(&a, 0, sizeof a);
    a.tp = tp;
    a.skip = l.one;
    int rc = launch_blend_node(a, 1, s);
    if (rc) return rc;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    RGS_CUDA_TRY(cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &nd));
    if (st != cudaStreamCaptureStatusActive || nd != 1 || !deps) {
        set_error("serve: the per-request blend is not the capture's last node");
        return RGS_ECUDA;
    }
    *node = deps[0];
    return RGS_OK;
}

int ceil_log2(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) ++b;
    return b;
}

// Enqueues the whole batch pipeline of one lane on `s` (captured into the lane's graph).
// record_ends: the blend cuts saturated runs back for a batched backward's replay.
int enqueue_batch(const rgs_gaussians& g, const TreeParams& tp, int K, int L, int slots, int64_t tiles_cap,
                  const LaneBufs& l, const BatchSlot* slots_host, const BatchHeader* hdr_host,
                  unsigned long long* status_host, cudaStream_t s, bool record_ends, const uint32_t** ival_out,
                  const BatchSlot* slots2_host, BlendNodes* nodes) {
    const int64_t N = g.n, P = N * slots;
    const bool grouped = slots2_host != nullptr;
    if (grouped && (!l.slots2 || !l.b.cnt_bin || record_ends || !nodes)) {
        set_error("serve: binning in groups needs a lane laid out for it, per-request blends, no recorded run ends");
        return RGS_EINVAL;
    }
    if (nodes && (record_ends || slots > kMaxSlots)) {
        set_error("serve: per-request blends record no run ends");
        return RGS_EINVAL;
    }
    RasterBuffers b = l.b;
    if (!grouped) b.cnt_bin = nullptr;   // one group: the projection counts every rank only
    unsigned long long* c = l.counters;
    unsigned long long* cb = c + kBatchBinCounter;
    int rc;
    RGS_CUDA_TRY(cudaMemcpyAsync(l.hdr, hdr_host, sizeof(BatchHeader), cudaMemcpyHostToDevice, s));
    RGS_CUDA_TRY(cudaMemcpyAsync(l.slots, slots_host, sizeof(BatchSlot) * slots, cudaMemcpyHostToDevice, s));
    if (grouped)
        RGS_CUDA_TRY(cudaMemcpyAsync(l.slots2, slots2_host, sizeof(BatchSlot) * slots, cudaMemcpyHostToDevice, s));
    RGS_CUDA_TRY(cudaMemsetAsync(c, 0, 8 * kBatchCounters, s));
    RGS_CUDA_TRY(cudaMemsetAsync(b.ranges, 0, sizeof(uint2) * tiles_cap * K, s));
    if (grouped) RGS_CUDA_TRY(cudaMemsetAsync(b.open, 0, (size_t)tiles_cap, s));
    if ((rc = launch_clip_table_batch(l.slots, l.hdr, tp, s))) return rc;
    if ((rc = launch_project_batch(g, l.slots, l.hdr, tp, b, c, s))) return rc;
    // compaction in (request, splat) order
    if ((rc = exclusive_scan_dev(b.cnt, b.vis_pos, &l.hdr->n_total, P, 1, nullptr, b.temp, b.temp_bytes, s)))
        return rc;
    compact_batch_kernel<<<grid_stride_blocks(), 256, 0, s>>>(b.cnt, b.vis_pos, b.dkey_lo, &l.hdr->n_total, P, b.skey, b.sid);
    RGS_CUDA_LAUNCH_CHECK();
    // (request, depth, index) order: LSD passes on the low depth bits, the float bits of
    // z, then the request
    uint32_t *ka = b.skey, *va = b.sid, *kb = b.skey_alt, *vb = b.sid_alt;
    auto sort = [&](int bits) -> int {
        bool alt = false;
        int r = radix_sort_pairs_dev(ka, va, kb, vb, &c[1], P, bits, b.temp, b.temp_bytes, s, &alt);
        if (!r && alt) {
            std::swap(ka, kb);
            std::swap(va, vb);
        }
        return r;
    };
    if ((rc = sort(16))) return rc;
    batch_key_kernel<<<grid_stride_blocks(), 256, 0, s>>>(b.dkey, va, N, &c[1], P, ka);
    RGS_CUDA_LAUNCH_CHECK();
    if ((rc = sort(31))) return rc;
    if (slots > 1) {
        batch_key_kernel<<<grid_stride_blocks(), 256, 0, s>>>(nullptr, va, N, &c[1], P, ka);
        RGS_CUDA_LAUNCH_CHECK();
        if ((rc = sort(ceil_log2(slots)))) return rc;
    }
    const uint32_t* sorted_ids = va;
    if ((rc = exclusive_scan_dev(grouped ? b.cnt_bin : b.cnt, b.ioff, &c[1], P, 2, sorted_ids, b.temp, b.temp_bytes,
                                 s)))
        return rc;
    check_capacity_kernel<<<1, 1, 0, s>>>(c, b.inst_cap, grouped);
    RGS_CUDA_LAUNCH_CHECK();
    if ((rc = launch_emit_batch(l.slots, l.hdr, tp, b, sorted_ids, P, N, c, s))) return rc;
    bool alt = false;
    const int key_bits = ceil_log2(tiles_cap) + L;
    if ((rc = radix_sort_pairs_dev(b.ikey, b.ival, b.ikey_alt, b.ival_alt, &c[4], b.inst_cap, key_bits, b.temp,
                                   b.temp_bytes, s, &alt)))
        return rc;
    const uint32_t* keys = alt ? b.ikey_alt : b.ikey;
    const uint32_t* ival = alt ? b.ival_alt : b.ival;
    if (ival_out) *ival_out = ival;
    if ((rc = launch_ranges_dev(keys, &c[4], b.inst_cap, b.ranges, s))) return rc;
    if (nodes) {
        nodes->ival = ival;
        for (int q = 0; q < slots; ++q)
            if ((rc = capture_blend_node(l, tp, s, &nodes->g1[q]))) return rc;
    } else if ((rc = launch_blend_batch(l.slots, l.hdr, tp, b.ranges, ival, b.rec, c, s, record_ends))) {
        return rc;
    }
    if (grouped) {
        // the second group: ranks [bin_lo, K) of the slots2 views in the tiles left open,
        // counted per visible pair in depth order (into vis_pos), emitted after the first
        // group's instances, sorted there (same key bits: the same buffer parity), blended
        // request by request in the open tiles
        if ((rc = launch_open_tables_batch(l.slots2, l.hdr, b.open, s))) return rc;
        if ((rc = launch_recount_batch(l.slots2, l.hdr, tp, b, sorted_ids, P, N, c, b.vis_pos, cb + 2, cb + 1, s)))
            return rc;
        check_group2_kernel<<<1, 1, 0, s>>>(c, b.inst_cap);
        RGS_CUDA_LAUNCH_CHECK();
        if ((rc = exclusive_scan_dev(b.vis_pos, b.ioff, &c[1], P, 0, nullptr, b.temp, b.temp_bytes, s))) return rc;
        RGS_CUDA_TRY(cudaMemsetAsync(c + 5, 0, 16, s));   // the emission's work queues
        if ((rc = launch_emit_batch(l.slots2, l.hdr, tp, b, sorted_ids, P, N, c, s, &c[4], true))) return rc;
        bool alt2 = false;
        if ((rc = radix_sort_pairs_dev(b.ikey, b.ival, b.ikey_alt, b.ival_alt, cb + 1, b.inst_cap, key_bits, b.temp,
                                       b.temp_bytes, s, &alt2, &c[4])))
            return rc;
        if (alt2 != alt) {
            set_error("serve: the binning groups' sorts end in different buffers");
            return RGS_EINVAL;
        }
        if ((rc = launch_ranges_dev(keys, cb + 1, b.inst_cap, b.ranges, s, &c[4]))) return rc;
        for (int q = 0; q < slots; ++q)
            if ((rc = capture_blend_node(l, tp, s, &nodes->g2[q]))) return rc;
    }
    RGS_CUDA_TRY(cudaMemcpyAsync(status_host, c, 8 * kBatchCounters, cudaMemcpyDeviceToHost, s));
    return RGS_OK;
}

namespace {

// ------------------------------------------------------------------ server state
using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

struct Request {
    uint64_t ticket;
    rgs_camera cam;
    ViewParams vp;
    float* out;
    int64_t tiles;
    int64_t pixels;
    int64_t exact_inst = -1;      // known after a batch holding it overflowed
    Clock::time_point t_submit;
    bool done = false;
    int status = RGS_OK;
    double latency_ms = 0;
    char err[160] = {0};
};

struct Lane {
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphExec_t exec2 = nullptr;     // the batch with binning in two groups of ranks
    cudaGraph_t graph[2] = {nullptr, nullptr};   // kept: their per-request blend nodes
    BlendNodes nodes[2];
    BatchSlot* slots2_host = nullptr;    // pinned: the second group's slot table
    cudaEvent_t done_ev = nullptr;
    char* mem = nullptr;
    LaneBufs bufs;
    BatchSlot* slots_host = nullptr;     // pinned
    BatchHeader* hdr_host = nullptr;     // pinned
    unsigned long long* status_host = nullptr;   // pinned [kBatchCounters]
    std::vector<Request*> inflight;
    bool busy = false;
};

}  // namespace
}  // namespace rgs

struct rgs_server {
    const rgs_kd* kd;
    rgs_gaussians g;
    rgs_render_opts opts;
    rgs_serve_config cfg;
    rgs::TreeParams tp;
    int device;
    int K, L;
    int64_t tiles_cap;      // per lane (batched) / per request (plain)
    int64_t inst_cap;
    std::vector<rgs::Lane> lanes;
    // plain mode
    void* plain_ws = nullptr;
    size_t plain_ws_bytes = 0;
    cudaStream_t plain_stream = nullptr;
    cudaEvent_t plain_ev = nullptr;
    // queue and tickets
    std::mutex mu;
    std::condition_variable cv;
    std::deque<rgs::Request*> queue;
    std::unordered_map<uint64_t, rgs::Request*> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool broken = false;
    bool hold = false;
    double inst_per_pixel = 16.0;   // running estimate for admission
    bool group_lanes = false;       // lanes laid out (and captured) for binning in two groups
    // measured tile instances (per visible splat, and in all), by resolution (width << 32 | height)
    std::unordered_map<uint64_t, std::pair<double, double>> inst_history;
    rgs_serve_stats stats;
    int64_t batched_requests = 0;
    std::thread worker;
    bool worker_timed_out = false;
};

namespace rgs {
namespace {

void finish(rgs_server* S, Request* r, int status, const char* why) {
    r->status = status;
    r->latency_ms = ms_since(r->t_submit);
    if (why) snprintf(r->err, sizeof r->err, "%s", why);
    r->done = true;
    if (status == RGS_OK) ++S->stats.completed;
    else if (status == RGS_EAGAIN) ++S->stats.cancelled;
    else ++S->stats.failed;
}

int64_t est_instances(const rgs_server* S, const Request* r) {
    if (r->exact_inst >= 0) return r->exact_inst;
    return (int64_t)(S->inst_per_pixel * 1.25 * (double)r->pixels) + 1024;
}

// Pops the next batch for a lane (caller holds S->mu).
void form_batch(rgs_server* S, std::vector<Request*>& batch) {
    int64_t tiles = 0, inst = 0, pix = 0;
    const int64_t max_pix = S->cfg.batch_max_pixels;
    while (!S->queue.empty() && (int)batch.size() < S->cfg.max_slots) {
        Request* r = S->queue.front();
        const int64_t e = est_instances(S, r);
        if (!batch.empty() && (tiles + r->tiles > S->tiles_cap || inst + e > S->inst_cap ||
                               (max_pix > 0 && pix + r->pixels > max_pix)))
            break;
        S->queue.pop_front();
        tiles += r->tiles;
        inst += e;
        pix += r->pixels;
        batch.push_back(r);
    }
}

uint64_t resolution_key(const Request* r) {
    return ((uint64_t)(uint32_t)r->cam.width << 32) | (uint32_t)r->cam.height;
}

// Whether a request bins its subsets in two groups of view ranks: the lanes allow it and
// the batches before measured enough instances (per visible splat, and in all) at its
// resolution (the rule of rgs_render_fwd's image-only forward, from the resolution's
// history), or the options or thresholds ask for it always.
bool wants_groups(const rgs_server* S, const Request* r) {
    if (!S->group_lanes) return false;
    if (S->opts.group_binning == 2 || (!(S->cfg.group_per_splat > 0.f) && !(S->cfg.group_min_instances > 0.f)))
        return true;
    const auto it = S->inst_history.find(resolution_key(r));
    return it != S->inst_history.end() && it->second.first >= (double)S->cfg.group_per_splat &&
           it->second.second >= (double)S->cfg.group_min_instances;
}

int launch_lane(rgs_server* S, Lane& ln, std::vector<Request*>& batch) {
    BatchHeader& h = *ln.hdr_host;
    memset(&h, 0, sizeof h);
    h.S = (int)batch.size();
    h.n_total = (unsigned long long)S->g.n * (unsigned long long)h.S;
    const int r1 = S->K / 8 > 1 ? S->K / 8 : 1;   // the first group's ranks, as rgs_render_fwd
    bool any_grouped = false;
    int64_t poff = 0, soff = 0, sbase = 0;
    uint32_t base = 0;
    for (int s = 0; s < h.S; ++s) {
        h.tile_base[s] = base;
        BatchSlot& a = ln.slots_host[s];
        a.vp = batch[s]->vp;
        a.vp.set_clip(ln.bufs.clip_plane + (size_t)s * kClipTable, ln.bufs.clip_margin + (size_t)s * kClipTable);
        a.image = batch[s]->out;
        a.tile_base = base;
        // grouped while the lane's group state has room for the request's tiles
        const bool grp = wants_groups(S, batch[s]) && sbase + batch[s]->tiles <= ln.bufs.group_tiles;
        a.state_base = (uint32_t)sbase;
        if (grp) sbase += batch[s]->tiles;
        a.vp.bin_lo = 0;
        a.vp.bin_hi = grp ? r1 : S->K;
        if (S->group_lanes) {
            BatchSlot& a2 = ln.slots2_host[s];
            a2 = a;
            a2.vp.bin_lo = grp ? r1 : S->K;   // none: every rank went with the first group
            a2.vp.bin_hi = S->K;
            a2.vp.set_open(ln.bufs.b.open_prefix + poff, ln.bufs.b.open_sat + soff);
            poff += (int64_t)a.vp.tiles_y * (a.vp.tiles_x + 1);
            soff += (int64_t)(a.vp.tiles_y + 1) * (a.vp.tiles_x + 1);
        }
        any_grouped |= grp;
        base += (uint32_t)batch[s]->tiles;
    }
    if (poff > ln.bufs.prefix_cap || soff > ln.bufs.sat_cap) {
        set_error("serve: open-tile tables exceed the lane's");
        return RGS_EOVERFLOW;
    }
    for (int s = h.S; s <= kMaxSlots; ++s) h.tile_base[s] = base;
    h.total_tiles = base;
    // each request's blend launches: its view, tiles and group; the unused slots' do nothing
    const BlendNodes& nd = ln.nodes[any_grouped ? 1 : 0];
    cudaGraphExec_t ex = any_grouped ? ln.exec2 : ln.exec;
    const LaneBufs& l = ln.bufs;
    for (int s = 0; s < S->cfg.max_slots; ++s) {
        for (int grp2 = 0; grp2 < (any_grouped ? 2 : 1); ++grp2) {
            const BatchSlot& sl = grp2 ? ln.slots2_host[s] : ln.slots_host[s];
            BlendNodeArgs a;
            memset(&a, 0, sizeof a);
            a.tp = S->tp;
            a.skip = l.one;
            unsigned grid = 1;
            if (s < h.S && (grp2 == 0 || sl.vp.bin_lo < S->K)) {
                a.vp = sl.vp;
                a.ival = nd.ival;
                a.rec = l.b.rec;
                a.ranges = l.b.ranges + (size_t)sl.tile_base * S->K;
                a.image = sl.image;
                a.r_begin = sl.vp.bin_lo;
                a.r_end = sl.vp.bin_hi;
                if (sl.vp.bin_lo > 0 || sl.vp.bin_hi < S->K) {   // a grouped request: its state
                    a.state = l.b.state + (size_t)sl.state_base * kTilePixels;
                    a.open = l.b.open + sl.tile_base;
                }
                a.skip = l.counters + 2;   // the overflow flag
                grid = (unsigned)((int64_t)sl.vp.tiles_x * sl.vp.tiles_y);
            }
            int rc = set_blend_node(ex, grp2 ? nd.g2[s] : nd.g1[s], a, grid);
            if (rc) return rc;
        }
    }
    RGS_CUDA_TRY(cudaGraphLaunch(ex, ln.stream));
    RGS_CUDA_TRY(cudaEventRecord(ln.done_ev, ln.stream));
    ln.inflight = batch;
    ln.busy = true;
    ++S->stats.batches;
    S->batched_requests += h.S;
    return RGS_OK;
}

// Lane finished (caller holds S->mu): settle its requests.
void complete_lane(rgs_server* S, Lane& ln) {
    const unsigned long long* st = ln.status_host;
    const bool overflow = st[2] != 0;
    const int n = (int)ln.inflight.size();
    if (st[2] == 2) {   // inconsistent group counts (not expected): nothing was written
        for (Request* r : ln.inflight)
            finish(S, r, RGS_EINVAL, "serve: the binning groups' instance counts disagree; batch not rendered");
    } else if (!overflow) {
        int64_t inst = 0, pix = 0;
        for (int s = 0; s < n; ++s) {
            finish(S, ln.inflight[s], RGS_OK, nullptr);
            const unsigned long long I = st[kBatchSlotCounters + 2 * s], V = st[kBatchSlotCounters + 2 * s + 1];
            inst += (int64_t)I;
            pix += ln.inflight[s]->pixels;
            if (V > 0) {
                const double r = (double)I / (double)V;
                auto it = S->inst_history.find(resolution_key(ln.inflight[s]));
                if (it == S->inst_history.end()) {
                    S->inst_history[resolution_key(ln.inflight[s])] = std::make_pair(r, (double)I);
                } else {
                    it->second.first = 0.7 * it->second.first + 0.3 * r;
                    it->second.second = 0.7 * it->second.second + 0.3 * (double)I;
                }
            }
        }
        if (pix > 0) S->inst_per_pixel = 0.8 * S->inst_per_pixel + 0.2 * ((double)inst / (double)pix);
    } else {
        // exact sizes are known now: requeue at the front, in order
        for (int s = n - 1; s >= 0; --s) {
            Request* r = ln.inflight[s];
            r->exact_inst = (int64_t)st[kBatchSlotCounters + 2 * s];
            if (n == 1 || r->exact_inst > S->inst_cap) {
                char why[160];
                snprintf(why, sizeof why, "serve: request needs %lld tile instances, a lane holds %lld",
                         (long long)r->exact_inst, (long long)S->inst_cap);
                finish(S, r, RGS_EOVERFLOW, why);
            } else {
                S->queue.push_front(r);
                ++S->stats.requeued;
            }
        }
    }
    ln.inflight.clear();
    ln.busy = false;
}

void fail_all(rgs_server* S, const char* why) {
    for (auto& ln : S->lanes) {
        for (Request* r : ln.inflight) finish(S, r, RGS_ECUDA, why);
        ln.inflight.clear();
    }
    for (Request* r : S->queue) finish(S, r, RGS_ECUDA, why);
    S->queue.clear();
    S->broken = true;
}

void worker_batched(rgs_server* S) {
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progress = false;
        for (auto& ln : S->lanes) {
            if (!ln.busy) continue;
            const cudaError_t e = cudaEventQuery(ln.done_ev);
            if (e == cudaSuccess) {
                complete_lane(S, ln);
                progress = true;
            } else if (e != cudaErrorNotReady) {
                fail_all(S, cudaGetErrorString(e));
                ln.busy = false;
            }
        }
        if (S->stop) break;
        if (!S->broken && !S->hold) {
            for (auto& ln : S->lanes) {
                if (ln.busy || S->queue.empty()) continue;
                std::vector<Request*> batch;
                form_batch(S, batch);
                if (batch.empty()) break;
                if (launch_lane(S, ln, batch) != RGS_OK) {
                    for (Request* r : batch) S->queue.push_front(r);
                    fail_all(S, "serve: graph launch failed");
                    break;
                }
                progress = true;
            }
        }
        if (!progress) {
            bool any_busy = false;
            for (auto& ln : S->lanes) any_busy |= ln.busy;
            // short naps while batches run; otherwise sleep until a submit or stop
            if (any_busy) S->cv.wait_for(lk, std::chrono::microseconds(20));
            else S->cv.wait_for(lk, std::chrono::milliseconds(50));
        }
    }
    // stopping: cancel the queue, wait (bounded) for the lanes
    for (Request* r : S->queue) finish(S, r, RGS_EAGAIN, "serve: cancelled (server destroyed)");
    S->queue.clear();
    const Clock::time_point t0 = Clock::now();
    for (;;) {
        bool any = false;
        for (auto& ln : S->lanes) {
            if (!ln.busy) continue;
            const cudaError_t e = cudaEventQuery(ln.done_ev);
            if (e == cudaErrorNotReady) any = true;
            else if (e == cudaSuccess) complete_lane(S, ln);
            else ln.busy = false;
        }
        if (!any) break;
        if (ms_since(t0) > 10000.0) {
            S->worker_timed_out = true;
            break;
        }
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(200));
        lk.lock();
    }
}

void worker_plain(rgs_server* S) {
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        if (S->stop) break;
        if (S->queue.empty() || S->broken || S->hold) {
            S->cv.wait_for(lk, std::chrono::milliseconds(50));
            continue;
        }
        Request* r = S->queue.front();
        S->queue.pop_front();
        ++S->stats.batches;
        ++S->batched_requests;
        lk.unlock();
        unsigned long long counts[2] = {0, 0};
        prof_suppress(true);
        int rc = render_fwd_into(S->kd, &S->g, &r->cam, &S->opts, nullptr, nullptr, r->out, nullptr, nullptr,
                                 S->plain_ws, S->plain_ws_bytes, S->plain_stream, counts);
        prof_suppress(false);
        std::string why = rc ? std::string(rgs_last_error()) : std::string();
        bool timed_out = false;
        if (rc == RGS_OK) {
            cudaError_t e = cudaEventRecord(S->plain_ev, S->plain_stream);
            const Clock::time_point t0 = Clock::now();
            while (e == cudaSuccess) {
                e = cudaEventQuery(S->plain_ev);
                if (e == cudaSuccess) break;
                if (e != cudaErrorNotReady) break;
                e = cudaSuccess;
                if (ms_since(t0) > 10000.0) {
                    timed_out = true;
                    break;
                }
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
            if (timed_out) {
                rc = RGS_ETIMEOUT;
                why = "serve: render did not finish within 10 s";
            } else if (e != cudaSuccess) {
                rc = RGS_ECUDA;
                why = cudaGetErrorString(e);
            }
        }
        lk.lock();
        finish(S, r, rc, rc ? why.c_str() : nullptr);
        if (rc == RGS_ECUDA || rc == RGS_ETIMEOUT) {
            fail_all(S, why.c_str());
            if (timed_out) S->worker_timed_out = true;
        }
    }
    for (Request* r : S->queue) finish(S, r, RGS_EAGAIN, "serve: cancelled (server destroyed)");
    S->queue.clear();
}

void worker_main(rgs_server* S) {
    cudaSetDevice(S->device);
    if (S->cfg.plain) worker_plain(S);
    else worker_batched(S);
}

void free_lane(Lane& ln) {
    if (ln.exec) cudaGraphExecDestroy(ln.exec);
    if (ln.exec2) cudaGraphExecDestroy(ln.exec2);
    for (cudaGraph_t gr : ln.graph)
        if (gr) cudaGraphDestroy(gr);
    if (ln.slots2_host) cudaFreeHost(ln.slots2_host);
    if (ln.done_ev) cudaEventDestroy(ln.done_ev);
    if (ln.stream) cudaStreamDestroy(ln.stream);
    if (ln.mem) cudaFree(ln.mem);
    if (ln.slots_host) cudaFreeHost(ln.slots_host);
    if (ln.hdr_host) cudaFreeHost(ln.hdr_host);
    if (ln.status_host) cudaFreeHost(ln.status_host);
    ln = Lane();
}

void free_server(rgs_server* S, bool leak_device) {
    if (!leak_device) {
        for (auto& ln : S->lanes) free_lane(ln);
        if (S->plain_ws) cudaFree(S->plain_ws);
        if (S->plain_ev) cudaEventDestroy(S->plain_ev);
        if (S->plain_stream) cudaStreamDestroy(S->plain_stream);
    }
    for (auto& kv : S->tickets) delete kv.second;
    delete S;
}

}  // namespace
}  // namespace rgs

using namespace rgs;

extern "C" {

void rgs_serve_default_config(rgs_serve_config* cfg) {
    if (!cfg) return;
    cfg->mem_budget_bytes = (size_t)8 << 30;
    cfg->max_slots = 8;
    cfg->lanes = 2;
    cfg->plain = 0;
    cfg->max_width = 4096;
    cfg->max_height = 4096;
    cfg->max_queue = 65536;
    cfg->inst_per_pixel = 16.f;
    cfg->group_per_splat = (float)kGroupInstancesPerSplat;
    cfg->group_min_instances = (float)kGroupMinInstances;
    cfg->batch_max_pixels = (int64_t)1 << 21;
}

}  // extern "C"

namespace rgs {
// Tiles of group state a lane keeps: two requests of the largest size (or fewer slots).
int64_t group_state_tiles(const rgs_serve_config* cfg) {
    const int64_t max_tiles =
        (int64_t)((cfg->max_width + kTile - 1) / kTile) * ((cfg->max_height + kTile - 1) / kTile);
    return max_tiles * (cfg->max_slots < 2 ? cfg->max_slots : 2);
}
}  // namespace rgs

extern "C" {

int rgs_serve_lane_bytes(const rgs_kd* kd, const rgs_gaussians* g, const rgs_serve_config* cfg,
                         int64_t instance_capacity, size_t* bytes) {
    int rc;
    if (!kd || !cfg || !bytes) { set_error("serve_lane_bytes: NULL argument"); return RGS_EINVAL; }
    if ((rc = check_gaussians(g))) return rc;
    if (cfg->max_slots < 1 || cfg->max_slots > kMaxSlots || cfg->max_width < 1 || cfg->max_height < 1 ||
        instance_capacity < 0) {
        set_error("serve_lane_bytes: invalid configuration");
        return RGS_EINVAL;
    }
    const int64_t max_tiles =
        (int64_t)((cfg->max_width + kTile - 1) / kTile) * ((cfg->max_height + kTile - 1) / kTile);
    *bytes = lane_layout(nullptr, g->n, cfg->max_slots, max_tiles * cfg->max_slots, 1 << kd->b.L, instance_capacity,
                         nullptr, false, (1 << kd->b.L) >= 4 ? group_state_tiles(cfg) : 0);
    return RGS_OK;
}

int rgs_serve_create(const rgs_kd* kd, const rgs_gaussians* g, const rgs_render_opts* opts, size_t mem_budget_bytes,
                     int max_slots, rgs_server** out) {
    rgs_serve_config cfg;
    rgs_serve_default_config(&cfg);
    cfg.mem_budget_bytes = mem_budget_bytes;
    cfg.max_slots = max_slots;
    return rgs_serve_create_ex(kd, g, opts, &cfg, out);
}

int rgs_serve_create_ex(const rgs_kd* kd, const rgs_gaussians* g, const rgs_render_opts* opts,
                        const rgs_serve_config* cfg, rgs_server** out) {
    int rc;
    if (!out) { set_error("serve_create: NULL out"); return RGS_EINVAL; }
    *out = nullptr;
    if (!kd || !cfg) { set_error("serve_create: NULL kd or config"); return RGS_EINVAL; }
    if ((rc = check_gaussians(g)) || (rc = check_opts(opts))) return rc;
    if (kd->b.L > kMaxRenderDepth) {
        set_error("serve_create: KD depth %d > %d", kd->b.L, kMaxRenderDepth);
        return RGS_EINVAL;
    }
    if (cfg->max_slots < 1 || cfg->max_slots > kMaxSlots || cfg->lanes < 1 || cfg->lanes > 4 ||
        cfg->max_width < 1 || cfg->max_width > 16384 || cfg->max_height < 1 || cfg->max_height > 16384 ||
        cfg->max_queue < 1 || !(cfg->inst_per_pixel > 0.f) || !(cfg->group_per_splat >= 0.f) ||
        !(cfg->group_min_instances >= 0.f) || cfg->batch_max_pixels < 0) {
        set_error("serve_create: need max_slots in [1,%d], lanes in [1,4], max size in [1,16384], max_queue >= 1, "
                  "inst_per_pixel > 0, group thresholds and batch_max_pixels >= 0", kMaxSlots);
        return RGS_EINVAL;
    }
    rgs_server* S = new (std::nothrow) rgs_server();
    if (!S) { set_error("serve_create: out of host memory"); return RGS_ENOMEM; }
    S->kd = kd;
    S->g = *g;
    S->opts = *opts;
    S->cfg = *cfg;
    memset(&S->stats, 0, sizeof S->stats);
    S->inst_per_pixel = cfg->inst_per_pixel;
    S->L = kd->b.L;
    S->K = 1 << kd->b.L;
    memset(&S->tp, 0, sizeof S->tp);
    S->tp.L = kd->b.L;
    for (int j = 0; j < S->K - 1; ++j) {
        S->tp.axis[j] = kd->b.axis[j];
        S->tp.split[j] = kd->b.split[j];
    }
    auto fail = [&](int code) {
        free_server(S, false);
        return code;
    };
    if (cudaGetDevice(&S->device) != cudaSuccess) { set_error("serve_create: no CUDA device"); return fail(RGS_ECUDA); }
    const int64_t max_tiles =
        (int64_t)((cfg->max_width + kTile - 1) / kTile) * ((cfg->max_height + kTile - 1) / kTile);
    if (cfg->plain) {
        // one workspace for rgs_render_fwd's path
        rgs_camera big;
        memset(&big, 0, sizeof big);
        big.viewmat[0] = big.viewmat[5] = big.viewmat[10] = big.viewmat[15] = 1.f;
        big.fx = big.fy = 1.f;
        big.width = cfg->max_width;
        big.height = cfg->max_height;
        big.near_z = 0.2f;
        size_t fixed = 0;
        if ((rc = rgs_render_workspace_size(kd, g, &big, opts, 1 << 20, &fixed))) return fail(rc);
        if (cfg->mem_budget_bytes < fixed) {
            set_error("serve_create: budget %zu below the %zu bytes of one %dx%d render", cfg->mem_budget_bytes, fixed,
                      cfg->max_width, cfg->max_height);
            return fail(RGS_EINVAL);
        }
        S->plain_ws_bytes = cfg->mem_budget_bytes;
        S->tiles_cap = max_tiles;
        S->inst_cap = (int64_t)((cfg->mem_budget_bytes - fixed) / 16) + (1 << 20);
        if (cudaMalloc(&S->plain_ws, S->plain_ws_bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("serve_create: cannot allocate %zu device bytes", S->plain_ws_bytes);
            return fail(RGS_ENOMEM);
        }
        if (cudaStreamCreateWithFlags(&S->plain_stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&S->plain_ev, cudaEventDisableTiming) != cudaSuccess) {
            set_error("serve_create: stream/event creation failed");
            return fail(RGS_ECUDA);
        }
    } else {
        const size_t lane_budget = cfg->mem_budget_bytes / (size_t)cfg->lanes;
        S->tiles_cap = max_tiles * cfg->max_slots;
        if (ceil_log2(S->tiles_cap) + S->L > 32) { set_error("serve_create: tile keys exceed 32 bits"); return fail(RGS_EINVAL); }
        S->group_lanes = opts->group_binning >= 1 && S->K >= 4;
        const int64_t gl = S->group_lanes ? group_state_tiles(cfg) : 0;
        const size_t fixed = lane_layout(nullptr, g->n, cfg->max_slots, S->tiles_cap, S->K, 0, nullptr, false, gl);
        const int64_t min_inst = (int64_t)1 << 16;
        if (lane_budget < fixed + (size_t)min_inst * 16) {
            set_error("serve_create: a lane needs at least %zu bytes (%zu given per lane)", fixed + (size_t)min_inst * 16,
                      lane_budget);
            return fail(RGS_EINVAL);
        }
        int64_t cap = (int64_t)((lane_budget - fixed) / 16);
        while (cap > min_inst &&
               lane_layout(nullptr, g->n, cfg->max_slots, S->tiles_cap, S->K, cap, nullptr, false, gl) > lane_budget)
            cap -= 64;
        if (cap > 0xFFFFFFFEll) cap = 0xFFFFFFFEll;
        S->inst_cap = cap;
        S->lanes.resize(cfg->lanes);
        for (auto& ln : S->lanes) {
            const size_t bytes = lane_layout(nullptr, g->n, cfg->max_slots, S->tiles_cap, S->K, cap, nullptr, false, gl);
            if (cudaMalloc(&ln.mem, bytes) != cudaSuccess) {
                cudaGetLastError();
                set_error("serve_create: cannot allocate %zu device bytes for a lane", bytes);
                return fail(RGS_ENOMEM);
            }
            lane_layout(ln.mem, g->n, cfg->max_slots, S->tiles_cap, S->K, cap, &ln.bufs, false, gl);
            if (cudaMallocHost(&ln.slots_host, sizeof(BatchSlot) * kMaxSlots) != cudaSuccess ||
                cudaMallocHost(&ln.slots2_host, sizeof(BatchSlot) * kMaxSlots) != cudaSuccess ||
                cudaMallocHost(&ln.hdr_host, sizeof(BatchHeader)) != cudaSuccess ||
                cudaMallocHost(&ln.status_host, 8 * kBatchCounters) != cudaSuccess ||
                cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ln.done_ev, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                set_error("serve_create: pinned memory, stream or event creation failed");
                return fail(RGS_ECUDA);
            }
            memset(ln.slots_host, 0, sizeof(BatchSlot) * kMaxSlots);
            memset(ln.slots2_host, 0, sizeof(BatchSlot) * kMaxSlots);
            memset(ln.hdr_host, 0, sizeof(BatchHeader));
            // capture the lane's batch pipeline once (and once binning in two groups)
            if ((rc = sort_prepare())) return fail(rc);
            if (cudaMemset(ln.bufs.one, 0xFF, 8) != cudaSuccess) {
                cudaGetLastError();
                set_error("serve_create: cannot initialise a lane");
                return fail(RGS_ECUDA);
            }
            for (int v = 0; v < (gl ? 2 : 1); ++v) {
                cudaGraph_t graph = nullptr;
                RGS_CUDA_TRY(cudaStreamBeginCapture(ln.stream, cudaStreamCaptureModeThreadLocal));
                prof_suppress(true);
                rc = enqueue_batch(S->g, S->tp, S->K, S->L, cfg->max_slots, S->tiles_cap, ln.bufs, ln.slots_host,
                                   ln.hdr_host, ln.status_host, ln.stream, false, nullptr,
                                   v ? ln.slots2_host : nullptr, &ln.nodes[v]);
                prof_suppress(false);
                const cudaError_t ec = cudaStreamEndCapture(ln.stream, &graph);
                if (rc || ec != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    if (!rc) set_error("serve_create: stream capture failed: %s", cudaGetErrorString(ec));
                    return fail(rc ? rc : RGS_ECUDA);
                }
                ln.graph[v] = graph;   // its blend nodes take each batch's arguments
                const cudaError_t ei = cudaGraphInstantiate(v ? &ln.exec2 : &ln.exec, graph, 0);
                if (ei != cudaSuccess) {
                    set_error("serve_create: graph instantiation failed: %s", cudaGetErrorString(ei));
                    return fail(RGS_ECUDA);
                }
            }
        }
    }
    S->stats.instance_capacity = S->inst_cap;
    try {
        S->worker = std::thread(worker_main, S);
    } catch (...) {
        set_error("serve_create: cannot start the scheduler thread");
        return fail(RGS_ENOMEM);
    }
    *out = S;
    return RGS_OK;
}

int rgs_serve_submit(rgs_server* S, const rgs_camera* cam, float* out_image, uint64_t* ticket) {
    int rc;
    if (!S || !out_image || !ticket) { set_error("serve_submit: NULL argument"); return RGS_EINVAL; }
    if ((rc = check_camera(cam))) return rc;
    if (cam->width > S->cfg.max_width || cam->height > S->cfg.max_height) {
        set_error("serve_submit: %dx%d exceeds the server's %dx%d", cam->width, cam->height, S->cfg.max_width,
                  S->cfg.max_height);
        return RGS_EINVAL;
    }
    Request* r = new (std::nothrow) Request();
    if (!r) { set_error("serve_submit: out of host memory"); return RGS_ENOMEM; }
    r->cam = *cam;
    r->out = out_image;
    TreeParams tp_unused;
    fill_view(S->kd, &S->g, cam, &S->opts, &r->vp, &tp_unused);
    r->tiles = (int64_t)r->vp.tiles_x * r->vp.tiles_y;
    r->pixels = (int64_t)cam->width * cam->height;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop || S->broken) {
            delete r;
            set_error("serve_submit: server is stopping or failed");
            return RGS_EAGAIN;
        }
        if ((int64_t)S->queue.size() >= S->cfg.max_queue) {
            delete r;
            set_error("serve_submit: queue full (%d requests)", S->cfg.max_queue);
            return RGS_EAGAIN;
        }
        r->ticket = S->next_ticket++;
        r->t_submit = Clock::now();
        S->tickets[r->ticket] = r;
        S->queue.push_back(r);
        ++S->stats.submitted;
        *ticket = r->ticket;
    }
    S->cv.notify_one();
    return RGS_OK;
}

int rgs_serve_poll(rgs_server* S, uint64_t ticket, int* done, double* latency_ms) {
    if (!S || !done) { set_error("serve_poll: NULL argument"); return RGS_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) {
        set_error("serve_poll: unknown ticket %llu", (unsigned long long)ticket);
        return RGS_EINVAL;
    }
    Request* r = it->second;
    if (!r->done) {
        *done = 0;
        return RGS_OK;
    }
    *done = 1;
    if (latency_ms) *latency_ms = r->latency_ms;
    const int status = r->status;
    if (status != RGS_OK) set_error("%s", r->err[0] ? r->err : "serve: request failed");
    S->tickets.erase(it);
    delete r;
    return status;
}

int rgs_serve_hold(rgs_server* S, int hold) {
    if (!S) { set_error("serve_hold: NULL server"); return RGS_EINVAL; }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->hold = hold != 0;
    }
    S->cv.notify_all();
    return RGS_OK;
}

int rgs_serve_stats_read(rgs_server* S, rgs_serve_stats* out) {
    if (!S || !out) { set_error("serve_stats: NULL argument"); return RGS_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    out->mean_batch = S->stats.batches ? (double)S->batched_requests / (double)S->stats.batches : 0.0;
    return RGS_OK;
}

int rgs_serve_destroy(rgs_server* S) {
    if (!S) return RGS_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    const bool timed_out = S->worker_timed_out;
    free_server(S, timed_out);
    if (timed_out) {
        set_error("serve_destroy: work on the GPU did not finish within 10 s; its buffers were left allocated");
        return RGS_ETIMEOUT;
    }
    return RGS_OK;
}

}  // extern "C"
