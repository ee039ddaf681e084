// Training over several views of one scene in one launch sequence (a batch of views per
// step, as the paper trains with a batch size per step, Sec. 4).
//
// Forward: the B views go through the batch pipeline of the render server (one projection
// of every (view, splat) pair, one compaction and depth sort, emission with global tile
// keys, one instance sort, one persistent blend over the batch's tiles; every count stays
// on the device), with the image-only culling of rgs_render_fwd and each saturated run cut
// back to what was staged.  The lists stay in the caller's workspace, stamped with a nonce.
// Backward: one persistent launch replays every view's runs through the flat form (the
// adjoint of Eq. 2, which Eq. 5 equals exactly) into per-(view, splat) 2D gradients, then
// each view's are pulled back through its projection into the shared parameter gradients.
// A view's arithmetic is that of rgs_render_fwd / rgs_render_bwd_flat, and its records,
// keys and tiles never mix with another's.
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "rgs_internal.cuh"

namespace rgs {
namespace {

__global__ void batch_stamp_kernel(unsigned long long* p, unsigned long long v) { *p = v; }

// Page-locked host copies of a batch's slot table, header and status (one set per thread).
struct BatchHost {
    BatchSlot* slots = nullptr;
    BatchHeader* hdr = nullptr;
    unsigned long long* status = nullptr;
    ~BatchHost() {
        if (slots) cudaFreeHost(slots);
        if (hdr) cudaFreeHost(hdr);
        if (status) cudaFreeHost(status);
    }
};
thread_local BatchHost g_host;

int host_buffers() {
    if (!g_host.slots) RGS_CUDA_TRY(cudaMallocHost(&g_host.slots, sizeof(BatchSlot) * kMaxSlots));
    if (!g_host.hdr) RGS_CUDA_TRY(cudaMallocHost(&g_host.hdr, sizeof(BatchHeader)));
    if (!g_host.status) RGS_CUDA_TRY(cudaMallocHost(&g_host.status, 8 * (kBatchCounters + 1)));
    return RGS_OK;
}

// What a forward left in a workspace: its arguments, the lanes' instance capacity, where
// the sorted payloads are, and the nonce it wrote into the workspace's header.
struct BatchStamp {
    const rgs_kd* kd;
    rgs_gaussians g;
    rgs_render_opts opts;
    std::vector<rgs_camera> cams;
    std::vector<const float*> images;
    size_t ws_bytes;
    int64_t inst_cap;
    int64_t I;
    bool alt;
    unsigned long long nonce;
};
std::mutex g_mu;
std::unordered_map<const void*, BatchStamp> g_stamps;

int check_batch(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cams, int B,
                const rgs_render_opts* opts, const float* const* images, void* workspace) {
    int rc;
    if (!kd || !cams || !images) { set_error("render_batch: NULL argument"); return RGS_EINVAL; }
    if (B < 1 || B > kMaxSlots) { set_error("render_batch: %d views not in [1, %d]", B, kMaxSlots); return RGS_EINVAL; }
    if ((rc = check_gaussians(g)) || (rc = check_opts(opts))) return rc;
    for (int b = 0; b < B; ++b) {
        if ((rc = check_camera(&cams[b]))) return rc;
        if (!images[b] || !aligned(images[b], 4)) { set_error("render_batch: image %d NULL or misaligned", b); return RGS_EINVAL; }
    }
    if (kd->b.L > kMaxRenderDepth) {
        set_error("render_batch: KD depth %d > %d (at most 64 subsets per render)", kd->b.L, kMaxRenderDepth);
        return RGS_EINVAL;
    }
    if (workspace && !aligned(workspace, 256)) { set_error("render_batch: workspace must be 256-byte aligned"); return RGS_EINVAL; }
    return RGS_OK;
}

struct BatchViews {
    TreeParams tp;
    ViewParams vp[kMaxSlots];
    int64_t tiles;   // sum over the views
};

void batch_views(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cams, int B,
                 const rgs_render_opts* opts, BatchViews* v) {
    v->tiles = 0;
    for (int b = 0; b < B; ++b) {
        fill_view(kd, g, &cams[b], opts, &v->vp[b], &v->tp);
        v->tiles += (int64_t)v->vp[b].tiles_x * v->vp[b].tiles_y;
    }
}

// The slot table and header of the batch in the page-locked host buffers.
void fill_slots(const BatchViews& v, int B, int64_t N, const LaneBufs& l, float* const* images,
                const float* const* grads) {
    BatchHeader& h = *g_host.hdr;
    memset(&h, 0, sizeof h);
    h.S = B;
    h.n_total = (unsigned long long)N * (unsigned long long)B;
    uint32_t base = 0;
    for (int b = 0; b < B; ++b) {
        BatchSlot& sl = g_host.slots[b];
        memset(&sl, 0, sizeof sl);
        sl.vp = v.vp[b];
        sl.vp.set_clip(l.clip_plane + (size_t)b * kClipTable, l.clip_margin + (size_t)b * kClipTable);
        sl.image = images[b];
        sl.grad = grads ? grads[b] : nullptr;
        sl.tile_base = base;
        h.tile_base[b] = base;
        base += (uint32_t)(v.vp[b].tiles_x * v.vp[b].tiles_y);
    }
    for (int b = B; b <= kMaxSlots; ++b) h.tile_base[b] = base;
    h.total_tiles = base;
}

// The lanes' buffers in a workspace of ws_bytes, with the largest instance capacity that fits.
int64_t carve_batch(void* workspace, size_t ws_bytes, int64_t N, int B, int64_t tiles, int K, LaneBufs* l) {
    int64_t lo = 0, hi = (int64_t)(ws_bytes / 16) + 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (lane_layout(nullptr, N, B, tiles, K, mid, nullptr, true) <= ws_bytes) lo = mid; else hi = mid - 1;
    }
    lane_layout((char*)workspace, N, B, tiles, K, lo, l, true);
    return lo;
}

// The batch forward into `workspace`; on success the stamp of its lists is registered.
int batch_forward(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cams, int B,
                  const rgs_render_opts* opts, float* const* images, void* workspace, size_t ws_bytes,
                  cudaStream_t s, const BatchViews& v) {
    const int K = 1 << kd->b.L, L = kd->b.L;
    const int64_t N = g->n;
    if (ceil_log2(v.tiles) + L > 32) { set_error("render_batch: tile keys of the batch exceed 32 bits"); return RGS_EINVAL; }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_stamps.erase(workspace);   // its lists are about to be replaced
    }
    const size_t fixed = lane_layout(nullptr, N, B, v.tiles, K, 0, nullptr, true);
    if (!workspace || ws_bytes < fixed) {
        set_required_workspace(lane_layout(nullptr, N, B, v.tiles, K, (int64_t)1 << 22, nullptr, true));
        set_error("render_batch: workspace of %zu bytes is smaller than the %zu needed before binning", ws_bytes, fixed);
        return RGS_EOVERFLOW;
    }
    int rc;
    if ((rc = host_buffers())) return rc;
    LaneBufs l;
    const int64_t cap = carve_batch(workspace, ws_bytes, N, B, v.tiles, K, &l);
    fill_slots(v, B, N, l, images, nullptr);
    const uint32_t* ival = nullptr;
    {
        ProfScope ps(ST_BATCH_FWD, s);
        rc = enqueue_batch(*g, v.tp, K, L, B, v.tiles, l, g_host.slots, g_host.hdr, g_host.status, s, true, &ival);
        if (rc) return rc;
    }
    RGS_CUDA_TRY(cudaStreamSynchronize(s));
    const unsigned long long* st = g_host.status;
    if (st[2]) {
        set_required_workspace(lane_layout(nullptr, N, B, v.tiles, K, (int64_t)st[0], nullptr, true));
        set_error("render_batch: %llu tile instances need a larger workspace", st[0]);
        return RGS_EOVERFLOW;
    }
    prof_add_host_counts((int64_t)st[0], (int64_t)st[1]);
    BatchStamp bs;
    bs.kd = kd;
    bs.g = *g;
    bs.opts = *opts;
    bs.cams.assign(cams, cams + B);
    bs.images.assign(images, images + B);
    bs.ws_bytes = ws_bytes;
    bs.inst_cap = cap;
    bs.I = (int64_t)st[4];
    bs.alt = ival == l.b.ival_alt;
    bs.nonce = next_nonce();
    batch_stamp_kernel<<<1, 1, 0, s>>>(l.header, bs.nonce);
    RGS_CUDA_LAUNCH_CHECK();
    std::lock_guard<std::mutex> lk(g_mu);
    g_stamps[workspace] = std::move(bs);
    return RGS_OK;
}

bool same_g(const rgs_gaussians& a, const rgs_gaussians& b) {
    return a.means == b.means && a.log_scales == b.log_scales && a.quats == b.quats &&
           a.opacity_logits == b.opacity_logits && a.sh == b.sh && a.n == b.n && a.sh_degree == b.sh_degree;
}

}  // namespace
}  // namespace rgs

using namespace rgs;

extern "C" {

int rgs_render_batch_fwd(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cams, int B,
                         const rgs_render_opts* opts, float* const* images, void* workspace, size_t ws_bytes,
                         void* stream) {
    int rc = check_batch(kd, g, cams, B, opts, images, workspace);
    if (rc) return rc;
    BatchViews v;
    batch_views(kd, g, cams, B, opts, &v);
    return batch_forward(kd, g, cams, B, opts, images, workspace, ws_bytes, (cudaStream_t)stream, v);
}

int rgs_render_batch_bwd(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cams, int B,
                         const rgs_render_opts* opts, float* const* images, const float* const* dL_dimages,
                         const rgs_gaussian_grads* grads, void* workspace, size_t ws_bytes, void* stream) {
    int rc = check_batch(kd, g, cams, B, opts, images, workspace);
    if (rc) return rc;
    if (!dL_dimages || !grads || !grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits ||
        !grads->sh) {
        set_error("render_batch_bwd: NULL argument");
        return RGS_EINVAL;
    }
    for (int b = 0; b < B; ++b)
        if (!dL_dimages[b]) { set_error("render_batch_bwd: dL/dimage %d is NULL", b); return RGS_EINVAL; }
    if (!aligned(grads->quats, 16)) { set_error("render_batch_bwd: grads->quats must be 16-byte aligned"); return RGS_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    BatchViews v;
    batch_views(kd, g, cams, B, opts, &v);
    const int K = 1 << kd->b.L;
    const int64_t N = g->n;
    // the lists of the forward with these arguments, if the workspace still holds them
    bool have = false;
    BatchStamp st;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_stamps.find(workspace);
        if (it != g_stamps.end()) {
            st = it->second;
            have = st.kd == kd && same_g(st.g, *g) && memcmp(&st.opts, opts, sizeof *opts) == 0 &&
                   (int)st.cams.size() == B && st.ws_bytes == ws_bytes &&
                   memcmp(st.cams.data(), cams, sizeof(rgs_camera) * B) == 0;
            for (int b = 0; have && b < B; ++b) have = st.images[b] == images[b];
        }
    }
    if ((rc = host_buffers())) return rc;
    if (have) {
        LaneBufs l;
        carve_batch(workspace, ws_bytes, N, B, v.tiles, K, &l);
        RGS_CUDA_TRY(cudaMemcpyAsync(g_host.status + kBatchCounters, l.header, 8, cudaMemcpyDeviceToHost, s));
        RGS_CUDA_TRY(cudaStreamSynchronize(s));
        have = g_host.status[kBatchCounters] == st.nonce;   // nothing overwrote the workspace since
    }
    if (!have) {   // re-derive the lists (and the images they blend)
        if ((rc = batch_forward(kd, g, cams, B, opts, images, workspace, ws_bytes, s, v))) return rc;
        std::lock_guard<std::mutex> lk(g_mu);
        st = g_stamps[workspace];
    }
    LaneBufs l;
    carve_batch(workspace, ws_bytes, N, B, v.tiles, K, &l);
    fill_slots(v, B, N, l, images, dL_dimages);
    RGS_CUDA_TRY(cudaMemcpyAsync(l.slots, g_host.slots, sizeof(BatchSlot) * B, cudaMemcpyHostToDevice, s));
    const uint32_t* ival = st.alt ? l.b.ival_alt : l.b.ival;
    {
        ProfScope ps(ST_BLEND_BWD, s);
        RGS_CUDA_TRY(cudaMemsetAsync(l.b.g2d, 0, sizeof(float4) * 3 * (size_t)N * B, s));
        if ((rc = launch_blend_bwd_batch(l.slots, l.hdr, v.tp, l.b.ranges, ival, l.b.rec, l.b.g2d, st.I, N * B,
                                         l.counters, s)))
            return rc;
    }
    ProfScope ps(ST_PROJECT_BWD, s);
    for (int b = 0; b < B; ++b) {
        RasterBuffers bb = l.b;
        bb.g2d = l.b.g2d + 3 * (size_t)N * b;
        if ((rc = launch_project_bwd(*g, *grads, v.vp[b], bb, s))) return rc;
    }
    // the page-locked slot table is rewritten by the next call: the copy above must be done
    RGS_CUDA_TRY(cudaStreamSynchronize(s));
    return RGS_OK;
}

}  // extern "C"
