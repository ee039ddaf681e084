// Tile binning, partial-map blending (Eq. 3-4 with the indicator of Eq. 6), the ordered
// merge (Eq. 5) and their adjoints.
//
// Instances.  After the visible splats are sorted by depth, each splat emits one
// instance per (subset N_k holding it, 16x16 tile its footprint may touch), keyed by
// (tile, view rank of k).  A stable radix sort on that key leaves every (tile, subset)
// run in depth order, which is the order of Eq. 3.  A warp emits the instances of 32
// consecutive splats cooperatively so that giant splats do not serialise one thread and
// the writes are contiguous.
//
// Blend.  One CTA per tile, one thread per pixel.  For each subset in view order the CTA
// walks the run in batches of 256 records staged in shared memory, every pixel applies
// the truncation tests and Eq. 6 (only for splats held by several subsets), and stops
// the subset once its transmittance drops below eps_T (block vote, and a warp vote to
// skip work).  The partial (C_k, T_k) is stored; the merge of Eq. 5 is accumulated on
// the fly, so the image costs no extra pass.
//
// Backward.  The adjoint of Eq. 5 gives dL/dC_k = g P_k and dL/dT_k = P_k <g, S_k> per
// pixel (P_k: transmittance in front of subset k, S_k: colour behind it).  Each subset
// is then replayed front to back from its stored partials: recomputing sigma and T
// exactly as the forward did, with A_i the colour accumulated up to and including pair i,
//   dC_k/dsigma_i = T_i c_i - (C_k - A_i)/(1 - sigma_i),   dT_k/dsigma_i = -T_k/(1 - sigma_i).
// A warp takes its record list 8 entries at a time: each lane replays its pixel and leaves
// two scalars per pair in shared memory, then each lane sums one record over one row of
// the warp's pixels and four lanes combine the rows.  Per-splat 2D gradients are summed
// across the CTA in shared memory and added to global memory with one vector reduction
// per float4.
#include <cuda_fp16.h>

#include "eft.cuh"
#include "footprint.cuh"
#include "rgs_internal.cuh"

namespace rgs {
namespace {

constexpr int kBlendThreads = kTilePixels;  // 256
// Resident CTAs per SM the blend kernels are compiled for (register budget 65536 / (256 x this)).
#ifndef RGS_BLEND_MIN_BLOCKS
#define RGS_BLEND_MIN_BLOCKS 3
#endif
constexpr float kNegHalfLog2e = -0.72134752044448170f;  // -0.5 * log2(e)
// The backward handles a warp's record list in stretches of kBwdSub entries: pixel by pixel,
// then record by record (rows padded to kBwdSubPad floats: conflict-free in both phases).
constexpr int kBwdSub = 16;
constexpr int kBwdSubPad = kBwdSub + 1;

// exp(-d2/2) as 2^(d2 * -0.5 log2 e) on the SFU (ex2.approx, ~2 ulp); the forward and
// the backward call the same function, so the backward sees the forward's sigma exactly.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------------------ emission
// One warp per depth-sorted splat; lanes take the splat's (subset, tile row) items, find
// the row's tile columns from the footprint (the same arithmetic as the count), and
// write the row's instances at the positions a warp prefix sum gives them.
// Writes from slot `pos` on the instances of an item's tiles [c0, c1] in row ty (subset
// `rank`, splat `id` at depth z) that the depth table or the binning group's open-tile
// table keeps; `first` is the global index of the row's first tile.
__device__ __forceinline__ void write_kept(const ViewParams& vp, const float* __restrict__ cull,
                                           const float2* __restrict__ chunk, uint32_t first, int ty, int c0, int c1,
                                           uint32_t rank, float z, uint32_t id, uint32_t pos,
                                           uint32_t* __restrict__ ikey, uint32_t* __restrict__ ival) {
    if (vp.open_prefix()) {
        for (int c = c0; c <= c1; ++c) {
            if (!tile_open(vp, ty, c)) continue;
            ikey[pos] = ((first + (uint32_t)c) << vp.L) | rank;
            ival[pos] = id;
            ++pos;
        }
        return;
    }
    for (int ch = c0 / kCullChunk; ch <= c1 / kCullChunk; ++ch) {
        const int lo = max(c0, ch * kCullChunk), hi = min(c1, ch * kCullChunk + kCullChunk - 1);
        const float2 mm = chunk[cull_chunk_index(vp, ty, ch, (int)rank)];
        if (z > mm.y) continue;
        const bool all = z <= mm.x;
        for (int c = lo; c <= hi; ++c) {
            if (!all && !keep_tile(cull, vp, ty, c, (int)rank, z)) continue;
            ikey[pos] = ((first + (uint32_t)c) << vp.L) | rank;
            ival[pos] = id;
            ++pos;
        }
    }
}

// The (subset, row) items of one splat, as the emission walks them.
struct SplatItems {
    Footprint f;
    unsigned long long m;
    float z;
    int nsub, ty0, rows, items;
};

template <int kMulti>
__device__ __forceinline__ SplatItems load_items(const ViewParams& vp, uint32_t id, const ushort4* __restrict__ rect,
                                                 const unsigned long long* __restrict__ mask,
                                                 const float4* __restrict__ rec, const float4* __restrict__ foot_side) {
    SplatItems s;
    const ushort4 r = rect[id];
    s.m = mask[id];
    const float4 r0 = rec[3 * (size_t)id], r1 = rec[3 * (size_t)id + 1], r2 = rec[3 * (size_t)id + 2];
    s.f = make_footprint(r0.x, r0.y, r1.x, r1.y, r1.z, r0.w, r1.w, vp);
    if (kMulti == 1 && foot_side) s.f.zr = foot_depth_radius(r2.w, foot_side[id].x);
    s.z = r2.w;
    s.ty0 = r.y;
    s.rows = (int)r.w - (int)r.y + 1;
    s.nsub = __popcll(s.m);
    s.items = s.nsub * s.rows;
    return s;
}

// One round of a splat's items, [it0, it0 + 32) (lane l takes item it0 + l): each lane
// finds its item's tile columns, a warp prefix sum places the items' runs from `base`,
// and (kWrite) the instances are written; returns the round's instance count (the same
// on every lane).  Without depth culling the warp writes the round's contiguous range
// together (lane l writes positions l, l + 32, ...: coalesced stores), finding each
// position's item by a forward scan of the run starts.  Global tile indices start at
// tile_base.  Every lane of the warp calls it.
template <int kMulti, bool kWrite>
__device__ __forceinline__ uint32_t emit_round(const ViewParams& vp, const TreeParams& tp, const int8_t* rank_of,
                                               uint32_t id, const SplatItems& s, int it0, uint32_t base,
                                               uint32_t tile_base,
                                               const float* __restrict__ cull, const float2* __restrict__ chunk,
                                               uint32_t* __restrict__ ikey, uint32_t* __restrict__ ival, int lane,
                                               uint32_t* s_start, uint32_t* s_key0) {
    const int it = it0 + lane;
    int c0 = 1, c1 = 0, ty = 0;
    uint32_t rank = 0;
    if (it < s.items) {
        int k;
        item_span<kMulti>(s.f, vp, tp, s.m, s.nsub, s.z, s.ty0, s.rows, it, ty, k, c0, c1);
        rank = (uint32_t)rank_of[k];
    }
    const uint32_t w = kept_tiles(cull, chunk, vp, ty, c0, c1, (int)rank, s.z);
    uint32_t incl = w;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (!kWrite) return total;
    const uint32_t first = tile_base + (uint32_t)(ty * vp.tiles_x);
    if (!cull && !vp.open_prefix()) {
        s_start[lane] = incl - w;
        s_key0[lane] = ((first + (uint32_t)c0) << vp.L) | rank;
        __syncwarp();
        int cur = 0;
        for (uint32_t o = (uint32_t)lane; o < total; o += 32) {
            while (cur < 31 && s_start[cur + 1] <= o) ++cur;   // runs of empty items share a start
            ikey[base + o] = s_key0[cur] + ((o - s_start[cur]) << vp.L);
            ival[base + o] = id;
        }
        __syncwarp();
    } else if (w) {
        write_kept(vp, cull, chunk, first, ty, c0, c1, rank, s.z, id, base + incl - w, ikey, ival);
    }
    return total;
}

// Instances of one splat (record id, first instance slot `base`), written by the calling
// warp round after round.
template <int kMulti>
__device__ __forceinline__ void emit_one(const ViewParams& vp, const TreeParams& tp, const int8_t* rank_of, uint32_t id,
                                         uint32_t base, uint32_t tile_base, const ushort4* __restrict__ rect,
                                         const unsigned long long* __restrict__ mask, const float4* __restrict__ rec,
                                         const float* __restrict__ cull, const float2* __restrict__ chunk,
                                         uint32_t* __restrict__ ikey, uint32_t* __restrict__ ival, int lane,
                                         uint32_t* s_start, uint32_t* s_key0, const float4* __restrict__ foot_side) {
    const SplatItems s = load_items<kMulti>(vp, id, rect, mask, rec, foot_side);
    for (int it0 = 0; it0 < s.items; it0 += 32)
        base += emit_round<kMulti, true>(vp, tp, rank_of, id, s, it0, base, tile_base, cull, chunk, ikey, ival, lane,
                                         s_start, s_key0);
}

// Deferred emission.  The near splats come first in depth order and are the largest, so a
// warp that took a group of 32 of them would emit them one after another long after the
// other warps finished.  The first launch therefore emits only the splats a lane handles
// alone and lists the others with their instance base; the second launch hands the list
// out with a stride of the number of warps, so that the heavy head of the list spreads
// over all of them.  A splat that finds the list full is emitted on the spot by its warp.
// Either way every instance lands at the position its count gives it.
struct EmitQueues {
    uint2* list;                   // [cap] (id, instance base) of the deferred splats
    unsigned long long* count;     // splats listed (may exceed cap: those were emitted on the spot)
    uint32_t cap;
};

// Instances of one small splat (at most kEmitThreadItems items), written by one thread.
constexpr int kEmitThreadItems = kSplatThreadItems;

template <int kMulti>
__device__ __forceinline__ void emit_thread(const ViewParams& vp, const TreeParams& tp, const int8_t* rank_of,
                                            uint32_t id, uint32_t pos,
                                            uint32_t tile_base, const Footprint& f, unsigned long long m, int nsub,
                                            float z, int ty0, int rows, int items, const float* __restrict__ cull,
                                            const float2* __restrict__ chunk, uint32_t* __restrict__ ikey,
                                            uint32_t* __restrict__ ival) {
    for (int it = 0; it < items; ++it) {
        int ty, k, c0, c1;
        item_span<kMulti>(f, vp, tp, m, nsub, z, ty0, rows, it, ty, k, c0, c1);
        const uint32_t rank = (uint32_t)rank_of[k];
        if (!rank_binned(vp, (int)rank) || c0 > c1) continue;
        const uint32_t first = tile_base + (uint32_t)(ty * vp.tiles_x);
        if (cull || vp.open_prefix()) {
            const uint32_t w = kept_tiles(cull, chunk, vp, ty, c0, c1, (int)rank, z);
            write_kept(vp, cull, chunk, first, ty, c0, c1, rank, z, id, pos, ikey, ival);
            pos += w;
            continue;
        }
        for (int c = c0; c <= c1; ++c) {
            ikey[pos] = ((first + (uint32_t)c) << vp.L) | rank;
            ival[pos] = id;
            ++pos;
        }
    }
}

// Emission of the depth-sorted visible splats, 32 per warp: a splat with few (subset,
// row) items is emitted by its own lane, the others by the whole warp in turn (the same
// split as the count in the projection).  kMulti selects the splats this launch emits:
// those in one subset (0) or those straddling several (1, with the clipping code); two
// launches cover all, each compiled for its own register budget.
template <int kMulti>
__global__ void __launch_bounds__(256)
emit_kernel(ViewParams vp, TreeParams tp, const uint32_t* __restrict__ sorted_ids, int64_t n_vis,
            const uint32_t* __restrict__ ioff, const ushort4* __restrict__ rect,
            const unsigned long long* __restrict__ mask, const float4* __restrict__ rec, const float* __restrict__ cull,
            const float2* __restrict__ chunk, uint32_t* __restrict__ ikey, uint32_t* __restrict__ ival,
            unsigned long long* __restrict__ queue, const float4* __restrict__ foot_side, EmitQueues q,
            const uint32_t* __restrict__ item_at, uint32_t* __restrict__ ibase) {
    __shared__ uint32_t s_start[8][32], s_key0[8][32];
    __shared__ TreeParams stp;
    __shared__ int8_t srank[64];
    stage_tree(tp, vp.rank_of, stp, srank);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // groups of 32 splats are claimed, two at a time (half the atomics on the one queue
    // counter), from a device counter: the near (large) splats come first in depth order, so
    // the heavy groups start first and spread over all warps
    for (;;) {
        unsigned long long gq = 0;
        if (lane == 0) gq = atomicAdd(queue, 1ull);
        const int64_t pc = (int64_t)__shfl_sync(0xffffffffu, gq, 0) * 64;
        if (pc >= n_vis) break;
      for (int half = 0; half < 2; ++half) {
        const int64_t p0 = pc + 32 * half;
        if (p0 >= n_vis) break;
        const int64_t p = p0 + lane;
        uint32_t id = 0, base = 0;
        int items = 0;
        if (p < n_vis) {
            id = sorted_ids[p];
            base = ioff[p];
            const ushort4 r = rect[id];
            const unsigned long long m = mask[id];
            const int rows = (int)r.w - (int)r.y + 1, nsub = __popcll(m);
            items = ((nsub > 1) == (kMulti == 1)) && box_open(vp, r) ? nsub * rows : 0;
            if (items > 0 && items <= kEmitThreadItems) {
                const float4 r0 = rec[3 * (size_t)id], r1 = rec[3 * (size_t)id + 1], r2 = rec[3 * (size_t)id + 2];
                Footprint f = make_footprint(r0.x, r0.y, r1.x, r1.y, r1.z, r0.w, r1.w, vp);
                if (kMulti == 1 && foot_side) f.zr = foot_depth_radius(r2.w, foot_side[id].x);
                emit_thread<kMulti>(vp, stp, srank, id, base, 0u, f, m, nsub, r2.w, r.y, rows, items, cull, chunk,
                                    ikey, ival);
            }
        }
        bool listed = false;
        if (item_at && items > kEmitThreadItems && item_at[id] != kNoItems) {
            ibase[id] = base;   // the count kept its items: emit_items_kernel writes them
            listed = true;
        }
        if (q.list) {
            // one atomic per warp: lanes take consecutive slots in lane order
            const bool mine = items > kEmitThreadItems && !listed;
            const unsigned bal = __ballot_sync(0xffffffffu, mine);
            if (bal) {
                unsigned long long first = 0;
                if (lane == 0) first = atomicAdd(q.count, (unsigned long long)__popc(bal));
                first = __shfl_sync(0xffffffffu, first, 0);
                const unsigned long long slot = first + (unsigned long long)__popc(bal & ((1u << lane) - 1u));
                if (mine && slot < q.cap) {
                    q.list[slot] = make_uint2(id, base);
                    listed = true;
                }
            }
        }
        unsigned big = __ballot_sync(0xffffffffu, items > kEmitThreadItems && !listed);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const uint32_t sid_ = __shfl_sync(0xffffffffu, id, src), sbase = __shfl_sync(0xffffffffu, base, src);
            emit_one<kMulti>(vp, stp, srank, sid_, sbase, 0u, rect, mask, rec, cull, chunk, ikey, ival, lane,
                             s_start[wib], s_key0[wib], foot_side);
        }
      }
    }
}

// The listed splats, one per warp: warp w of the grid's W takes entries w, w + W, ...
template <int kMulti>
__global__ void __launch_bounds__(256, 2)
emit_listed_kernel(ViewParams vp, TreeParams tp, EmitQueues q, const ushort4* __restrict__ rect,
                   const unsigned long long* __restrict__ mask, const float4* __restrict__ rec,
                   const float* __restrict__ cull, const float2* __restrict__ chunk, uint32_t* __restrict__ ikey,
                   uint32_t* __restrict__ ival, const float4* __restrict__ foot_side) {
    __shared__ uint32_t s_start[8][32], s_key0[8][32];
    __shared__ TreeParams stp;
    __shared__ int8_t srank[64];
    stage_tree(tp, vp.rank_of, stp, srank);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned long long n = *q.count < q.cap ? *q.count : q.cap;
    const unsigned long long W = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long e = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + wib; e < n; e += W) {
        const uint2 it = q.list[e];
        emit_one<kMulti>(vp, stp, srank, it.x, it.y, 0u, rect, mask, rec, cull, chunk, ikey, ival, lane,
                         s_start[wib], s_key0[wib], foot_side);
    }
}

// The items the count kept, 32 per warp round (lane l takes entry q0 + l): each lane
// reads its item's record, the warp places the items' instance runs in one virtual range
// by a prefix sum and writes it together (lane l writes positions l, l + 32, ...), each
// position going to its item's run at that splat's first instance plus the item's offset.
// Items of one splat are consecutive entries with consecutive runs, so the stores stay
// contiguous within a splat.
__global__ void __launch_bounds__(256)
emit_items_kernel(ViewParams vp, const uint4* __restrict__ items, const uint32_t* __restrict__ first,
                  const unsigned long long* __restrict__ n_items, uint32_t cap, const uint32_t* __restrict__ ibase,
                  const float4* __restrict__ rec, const float* __restrict__ cull, const float2* __restrict__ chunk,
                  uint32_t* __restrict__ ikey, uint32_t* __restrict__ ival) {
    __shared__ uint32_t s_start[8][32], s_key0[8][32], s_dst[8][32], s_id[8][32];
    __shared__ int8_t srank[64];
    for (int k = threadIdx.x; k < 64; k += blockDim.x) srank[k] = vp.rank_of[k];
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned long long taken = *n_items;
    const unsigned long long n = taken < cap ? taken : cap;
    const unsigned long long stride = (unsigned long long)gridDim.x * (blockDim.x >> 5) * 32;
    for (unsigned long long q0 = ((unsigned long long)blockIdx.x * (blockDim.x >> 5) + wib) * 32; q0 < n;
         q0 += stride) {
        const unsigned long long q = q0 + lane;
        uint32_t id = kNoItems, w = 0, dst = 0, key0 = 0, rank = 0;
        int ty = 0, c0 = 1, c1 = 0;
        float z = 0.f;
        if (q < n) {
            const uint4 r = items[q];
            id = r.x;
            if (id != kNoItems) {
                c0 = (int)(int16_t)(r.z & 0xFFFFu);
                c1 = (int)(int16_t)(r.z >> 16);
                ty = (int)(r.w & 0xFFFFu);
                rank = (uint32_t)srank[r.w >> 16];
                if (cull) z = rec[3 * (size_t)id + 2].w;
                w = kept_tiles(cull, chunk, vp, ty, c0, c1, (int)rank, z);
                if (w) dst = ibase[id] + (first ? first[q] : r.y);
                key0 = (((uint32_t)(ty * vp.tiles_x) + (uint32_t)c0) << vp.L) | rank;
            }
        }
        uint32_t incl = w;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (!cull && !vp.open_prefix()) {
            s_start[wib][lane] = incl - w;
            s_key0[wib][lane] = key0;
            s_dst[wib][lane] = dst;
            s_id[wib][lane] = id;
            __syncwarp();
            int cur = 0;
            for (uint32_t o = (uint32_t)lane; o < total; o += 32) {
                while (cur < 31 && s_start[wib][cur + 1] <= o) ++cur;   // runs of empty items share a start
                const uint32_t off = o - s_start[wib][cur];
                ikey[s_dst[wib][cur] + off] = s_key0[wib][cur] + (off << vp.L);
                ival[s_dst[wib][cur] + off] = s_id[wib][cur];
            }
            __syncwarp();
        } else if (w) {
            write_kept(vp, cull, chunk, (uint32_t)(ty * vp.tiles_x), ty, c0, c1, rank, z, id, dst, ikey, ival);
        }
    }
}

// Open-tile table of a binning group: per tile row, the number of open tiles before each
// column (tiles_x + 1 entries); one warp per row.
__device__ __forceinline__ void open_prefix_row(const uint8_t* __restrict__ open_row, int tiles_x,
                                                uint32_t* __restrict__ out, int lane) {
    uint32_t run = 0;
    for (int c0 = 0; c0 < tiles_x; c0 += 32) {
        const int c = c0 + lane;
        const bool o = c < tiles_x && open_row[c] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, o);
        if (c < tiles_x) out[c] = run + (uint32_t)__popc(bal & ((1u << lane) - 1u));
        run += (uint32_t)__popc(bal);
    }
    if (lane == 0) out[tiles_x] = run;
}

__global__ void __launch_bounds__(256)
open_prefix_kernel(const uint8_t* __restrict__ open, int tiles_x, int tiles_y, uint32_t* __restrict__ prefix) {
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= tiles_y) return;
    open_prefix_row(open + (size_t)row * tiles_x, tiles_x, prefix + (size_t)row * (tiles_x + 1), lane);
}

// Summed-area table of the open tiles from the per-row prefixes: one thread per column
// boundary x, down the rows.
__device__ __forceinline__ void open_sat_col(const uint32_t* __restrict__ prefix, int tiles_x, int tiles_y,
                                             uint32_t* __restrict__ sat, int x) {
    const size_t W1 = (size_t)tiles_x + 1;
    uint32_t acc = 0;
    sat[x] = 0u;
    for (int y = 0; y < tiles_y; ++y) {
        acc += prefix[(size_t)y * W1 + x];
        sat[(size_t)(y + 1) * W1 + x] = acc;
    }
}

__global__ void __launch_bounds__(256)
open_sat_kernel(const uint32_t* __restrict__ prefix, int tiles_x, int tiles_y, uint32_t* __restrict__ sat) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x > tiles_x) return;
    open_sat_col(prefix, tiles_x, tiles_y, sat, x);
}

// The same tables for every request of a batch (slot blockIdx.y; the open flags of its
// tiles from its tile_base; its tables where its view points), grid-stride over the rows
// and the column boundaries.
__global__ void __launch_bounds__(256)
open_prefix_batch_kernel(const BatchSlot* __restrict__ slots, const BatchHeader* __restrict__ hdr,
                         const uint8_t* __restrict__ open) {
    const int sl = blockIdx.y;
    if (sl >= hdr->S) return;
    const ViewParams& vp = slots[sl].vp;
    const int tiles_x = vp.tiles_x, tiles_y = vp.tiles_y;
    const uint8_t* o = open + hdr->tile_base[sl];
    uint32_t* prefix = const_cast<uint32_t*>(vp.open_prefix());
    const int lane = threadIdx.x & 31;
    for (int row = blockIdx.x * 8 + (threadIdx.x >> 5); row < tiles_y; row += gridDim.x * 8)
        open_prefix_row(o + (size_t)row * tiles_x, tiles_x, prefix + (size_t)row * (tiles_x + 1), lane);
}

__global__ void __launch_bounds__(256)
open_sat_batch_kernel(const BatchSlot* __restrict__ slots, const BatchHeader* __restrict__ hdr) {
    const int sl = blockIdx.y;
    if (sl >= hdr->S) return;
    const ViewParams& vp = slots[sl].vp;
    uint32_t* sat = const_cast<uint32_t*>(vp.open_sat());
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x <= vp.tiles_x; x += gridDim.x * blockDim.x)
        open_sat_col(vp.open_prefix(), vp.tiles_x, vp.tiles_y, sat, x);
}

// Copies the batch's view parameters into shared memory (the whole block).
__device__ __forceinline__ void load_batch_views(const BatchSlot* __restrict__ slots, int S, ViewParams* svp) {
    constexpr int kWords = (int)(sizeof(ViewParams) / 4);
    for (int w = threadIdx.x; w < S * kWords; w += blockDim.x) {
        const int sl = w / kWords, o = w - sl * kWords;
        reinterpret_cast<uint32_t*>(&svp[sl])[o] = reinterpret_cast<const uint32_t*>(&slots[sl].vp)[o];
    }
    __syncthreads();
}

// Count of a later binning group (the view's rank range and open-tile table) for every
// visible splat, in depth order: cnt_out[p] for the splat at depth position p; the group's
// total is added to *total.  A splat of few items is counted by its lane from its
// footprint; a splat whose items the count kept is counted by the warp from its item
// records, whose first-instance offsets are rewritten for this group; other splats by the
// warp from their footprint.  Groups of 32 splats are claimed from *queue (zeroed
// beforehand).  kBatch: the splats are a batch's (slot * N + i), each counted in its slot's
// view (slots[s].vp), *n_dev of them (at most n_vis), nothing when the overflow flag is set;
// else one view, vp1, and n_vis splats.
template <bool kBatch>
__global__ void __launch_bounds__(256)
recount_kernel(ViewParams vp1, const BatchSlot* __restrict__ slots, const BatchHeader* __restrict__ hdr, int64_t N,
               TreeParams tp, const uint32_t* __restrict__ sorted_ids, int64_t n_vis,
               const unsigned long long* __restrict__ n_dev, const unsigned long long* __restrict__ overflow,
               const ushort4* __restrict__ rect, const unsigned long long* __restrict__ mask,
               const float4* __restrict__ rec, const uint32_t* __restrict__ item_at, uint4* __restrict__ items,
               uint32_t item_cap, uint32_t* __restrict__ cnt_out, unsigned long long* __restrict__ queue,
               unsigned long long* __restrict__ total) {
    __shared__ ViewParams svp[kBatch ? kMaxSlots : 1];
    __shared__ TreeParams stp;
    __shared__ int8_t srank_unused[64];
    if (kBatch) {
        if (*overflow) return;   // the batch is discarded
        load_batch_views(slots, hdr->S, svp);
        const unsigned long long nv = *n_dev;
        if (nv < (unsigned long long)n_vis) n_vis = (int64_t)nv;
    } else {
        constexpr int kWords = (int)(sizeof(ViewParams) / 4);
        for (int w = threadIdx.x; w < kWords; w += blockDim.x)
            reinterpret_cast<uint32_t*>(&svp[0])[w] = reinterpret_cast<const uint32_t*>(&vp1)[w];
    }
    stage_tree(tp, vp1.rank_of, stp, srank_unused);   // the views' ranks: svp[slot].rank_of
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long gq = 0;
        if (lane == 0) gq = atomicAdd(queue, 1ull);
        const int64_t p0 = (int64_t)__shfl_sync(0xffffffffu, gq, 0) * 32;
        if (p0 >= n_vis) break;
        const int64_t p = p0 + lane;
        uint32_t id = 0, count = 0;
        int nitems = 0, slot = 0;
        if (p < n_vis) {
            id = sorted_ids[p];
            if (kBatch) slot = (int)(id / (uint64_t)N);
            const ViewParams& vp = svp[slot];
            const ushort4 r = rect[id];
            const int rows = (int)r.w - (int)r.y + 1;
            nitems = box_open(vp, r) ? __popcll(mask[id]) * rows : 0;   // no open tile: nothing
            if (nitems <= kSplatThreadItems) {
                const SplatItems si = load_items<-1>(vp, id, rect, mask, rec, nullptr);
                for (int it = 0; it < nitems; ++it) {
                    int ty, k, c0, c1;
                    item_span<-1>(si.f, vp, stp, si.m, si.nsub, si.z, si.ty0, si.rows, it, ty, k, c0, c1);
                    count += kept_tiles(nullptr, nullptr, vp, ty, c0, c1, vp.rank_of[k], si.z);
                }
            }
        }
        unsigned big = __ballot_sync(0xffffffffu, nitems > kSplatThreadItems);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const uint32_t sid = __shfl_sync(0xffffffffu, id, src);
            const int sitems = __shfl_sync(0xffffffffu, nitems, src);
            const ViewParams& vp = svp[__shfl_sync(0xffffffffu, slot, src)];
            const uint32_t at = item_at ? item_at[sid] : kNoItems;
            SplatItems si;
            if (at == kNoItems) si = load_items<-1>(vp, sid, rect, mask, rec, nullptr);
            uint32_t acc = 0;
            for (int it0 = 0; it0 < sitems; it0 += 32) {
                const int it = it0 + lane;
                uint32_t w = 0;
                if (it < sitems) {
                    int ty, k, c0, c1;
                    if (at != kNoItems) {
                        const uint4 rc = items[at + it];
                        c0 = (int)(int16_t)(rc.z & 0xFFFFu);
                        c1 = (int)(int16_t)(rc.z >> 16);
                        ty = (int)(rc.w & 0xFFFFu);
                        k = (int)(rc.w >> 16);
                    } else {
                        item_span<-1>(si.f, vp, stp, si.m, si.nsub, si.z, si.ty0, si.rows, it, ty, k, c0, c1);
                    }
                    w = kept_tiles(nullptr, nullptr, vp, ty, c0, c1, vp.rank_of[k], 0.f);
                }
                uint32_t incl = w;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (at != kNoItems && it < sitems) items[at + it].y = acc + incl - w;
                acc += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == src) count = acc;
        }
        if (p < n_vis) cnt_out[p] = count;
        unsigned long long c64 = count;
        for (int o = 16; o > 0; o >>= 1) c64 += __shfl_xor_sync(0xffffffffu, c64, o);
        if (lane == 0 && c64) atomicAdd(total, c64);
    }
}

// Batch emission: sorted ids are slot * N + i, so each lane takes its splat's view from
// the block's shared copy of the slot table; the same thread / warp split as emit_kernel.
// Each view's binning group (rank range, open-tile tables) selects what is written;
// inst_base (nullable): the group's instances start at that index (a device value).
template <int kMulti>
__global__ void __launch_bounds__(256)
emit_batch_kernel(const BatchSlot* __restrict__ slots, const BatchHeader* __restrict__ hdr, TreeParams tp,
                  const uint32_t* __restrict__ sorted_ids, int64_t n_cap, int64_t N,
                  unsigned long long* __restrict__ counters, const uint32_t* __restrict__ ioff,
                  const ushort4* __restrict__ rect, const unsigned long long* __restrict__ mask,
                  const float4* __restrict__ rec, uint32_t* __restrict__ ikey, uint32_t* __restrict__ ival,
                  const uint32_t* __restrict__ item_at, uint32_t* __restrict__ ibase,
                  const unsigned long long* __restrict__ inst_base) {
    if (counters[2]) return;   // overflow: the batch is discarded
    if (inst_base) {
        const unsigned long long b0 = *inst_base;
        ikey += b0;
        ival += b0;
    }
    __shared__ ViewParams svp[kMaxSlots];
    __shared__ uint32_t sbase[kMaxSlots];
    const int S = hdr->S;
    if ((int)threadIdx.x < S) sbase[threadIdx.x] = hdr->tile_base[threadIdx.x];
    load_batch_views(slots, S, svp);
    const unsigned long long nv = counters[1];
    const int64_t n = nv < (unsigned long long)n_cap ? (int64_t)nv : n_cap;
    __shared__ uint32_t s_start[8][32], s_key0[8][32];
    __shared__ TreeParams stp;
    __shared__ int8_t srank_unused[64];
    stage_tree(tp, svp[0].rank_of, stp, srank_unused);   // ranks differ per request: svp[slot].rank_of
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned long long* queue = &counters[5 + kMulti];   // zeroed with the batch's counters
    for (;;) {
        // two groups of 32 per claim: half the atomics on the one queue counter
        unsigned long long gq = 0;
        if (lane == 0) gq = atomicAdd(queue, 1ull);
        const int64_t pc = (int64_t)__shfl_sync(0xffffffffu, gq, 0) * 64;
        if (pc >= n) break;
      for (int half = 0; half < 2; ++half) {
        const int64_t p0 = pc + 32 * half;
        if (p0 >= n) break;
        const int64_t p = p0 + lane;
        uint32_t id = 0, base = 0;
        int items = 0, slot = 0;
        if (p < n) {
            id = sorted_ids[p];
            base = ioff[p];
            slot = (int)(id / (uint64_t)N);
            const ushort4 r = rect[id];
            const unsigned long long m = mask[id];
            const int rows = (int)r.w - (int)r.y + 1, nsub = __popcll(m);
            items = ((nsub > 1) == (kMulti == 1)) && box_open(svp[slot], r) ? nsub * rows : 0;
            if (items > 0 && items <= kEmitThreadItems) {
                const ViewParams& vp = svp[slot];
                const float4 r0 = rec[3 * (size_t)id], r1 = rec[3 * (size_t)id + 1], r2 = rec[3 * (size_t)id + 2];
                const Footprint f = make_footprint(r0.x, r0.y, r1.x, r1.y, r1.z, r0.w, r1.w, vp);
                emit_thread<kMulti>(vp, stp, vp.rank_of, id, base, sbase[slot], f, m, nsub, r2.w, r.y, rows, items,
                                    nullptr, nullptr, ikey, ival);
            }
        }
        // a splat whose items the projection kept: emit_items_batch_kernel writes them
        const bool kept = item_at && items > kEmitThreadItems && item_at[id] != kNoItems;
        if (kept) ibase[id] = base;
        unsigned big = __ballot_sync(0xffffffffu, items > kEmitThreadItems && !kept);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const uint32_t sid_ = __shfl_sync(0xffffffffu, id, src), sb = __shfl_sync(0xffffffffu, base, src);
            const int ss = __shfl_sync(0xffffffffu, slot, src);
            emit_one<kMulti>(svp[ss], stp, svp[ss].rank_of, sid_, sb, sbase[ss], rect, mask, rec, nullptr, nullptr,
                             ikey, ival, lane, s_start[wib], s_key0[wib], nullptr);
        }
      }
    }
}

// The batch's kept items, as emit_items_kernel: record ids are slot * N + i, so each lane
// takes its item's view (tile columns, subset ranks, binning group) and tile base from the
// block's shared copy of the slot table.  open_tables: the views carry open-tile tables
// (a later binning group: each lane writes its item's open tiles, below the group's count
// *n_group_dev); inst_base as emit_batch_kernel.
__global__ void __launch_bounds__(256)
emit_items_batch_kernel(const BatchSlot* __restrict__ slots, const BatchHeader* __restrict__ hdr,
                        const uint4* __restrict__ items, const unsigned long long* __restrict__ n_items,
                        uint32_t cap, const uint32_t* __restrict__ ibase, int64_t N,
                        const unsigned long long* __restrict__ counters, uint32_t* __restrict__ ikey,
                        uint32_t* __restrict__ ival, const unsigned long long* __restrict__ inst_base,
                        bool open_tables, const unsigned long long* __restrict__ n_group_dev) {
    if (counters[2]) return;   // overflow: the batch is discarded
    if (inst_base) {
        const unsigned long long b0 = *inst_base;
        ikey += b0;
        ival += b0;
    }
    const unsigned long long n_group = n_group_dev ? *n_group_dev : ~0ull;
    __shared__ ViewParams svp[kMaxSlots];
    __shared__ uint32_t sbase[kMaxSlots];
    __shared__ uint32_t s_start[8][32], s_key0[8][32], s_dst[8][32], s_id[8][32];
    const int S = hdr->S;
    if ((int)threadIdx.x < S) sbase[threadIdx.x] = hdr->tile_base[threadIdx.x];
    load_batch_views(slots, S, svp);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned long long taken = *n_items;
    const unsigned long long n = taken < cap ? taken : cap;
    const unsigned long long stride = (unsigned long long)gridDim.x * (blockDim.x >> 5) * 32;
    const int L = svp[0].L;
    for (unsigned long long q0 = ((unsigned long long)blockIdx.x * (blockDim.x >> 5) + wib) * 32; q0 < n;
         q0 += stride) {
        const unsigned long long q = q0 + lane;
        uint32_t id = kNoItems, w = 0, dst = 0, key0 = 0, rank = 0;
        int ty = 0, c0 = 1, c1 = 0, slot = 0;
        if (q < n) {
            const uint4 r = items[q];
            id = r.x;
            if (id != kNoItems) {
                c0 = (int)(int16_t)(r.z & 0xFFFFu);
                c1 = (int)(int16_t)(r.z >> 16);
                ty = (int)(r.w & 0xFFFFu);
                const int k = (int)(r.w >> 16);
                slot = (int)(id / (uint64_t)N);
                const ViewParams& vp = svp[slot];
                rank = (uint32_t)vp.rank_of[k];
                w = kept_tiles(nullptr, nullptr, vp, ty, c0, c1, (int)rank, 0.f);
                if (w) dst = ibase[id] + r.y;
                key0 = ((sbase[slot] + (uint32_t)(ty * vp.tiles_x) + (uint32_t)c0) << L) | rank;
            }
        }
        if (open_tables) {   // uniform: the kept tiles of each item are not contiguous
            // (a record of a splat this group passes over has no open tile in its span, so
            // its stale base is never used; the group's count bounds the writes regardless)
            if (w && (unsigned long long)dst + w > n_group) w = 0;
            if (w) {
                const ViewParams& vp = svp[slot];
                write_kept(vp, nullptr, nullptr, sbase[slot] + (uint32_t)(ty * vp.tiles_x), ty, c0, c1, rank, 0.f, id,
                           dst, ikey, ival);
            }
            continue;
        }
        uint32_t incl = w;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        s_start[wib][lane] = incl - w;
        s_key0[wib][lane] = key0;
        s_dst[wib][lane] = dst;
        s_id[wib][lane] = id;
        __syncwarp();
        int cur = 0;
        for (uint32_t o = (uint32_t)lane; o < total; o += 32) {
            while (cur < 31 && s_start[wib][cur + 1] <= o) ++cur;   // runs of empty items share a start
            const uint32_t off = o - s_start[wib][cur];
            ikey[s_dst[wib][cur] + off] = s_key0[wib][cur] + (off << L);
            ival[s_dst[wib][cur] + off] = s_id[wib][cur];
        }
        __syncwarp();
    }
}

// (min, max) of the forward depth table over each run of kCullChunk tiles of a row.
__global__ void cull_chunk_kernel(ViewParams vp, const float* __restrict__ cull, float2* __restrict__ chunk) {
    const int nch = cull_nchunk(vp);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)vp.tiles_y * nch * vp.K;
    if (i >= total) return;
    const int rank = (int)(i % vp.K);
    const int ch = (int)((i / vp.K) % nch);
    const int ty = (int)(i / ((int64_t)vp.K * nch));
    const int c_lo = ch * kCullChunk, c_hi = min(vp.tiles_x, (ch + 1) * kCullChunk);
    float lo = __int_as_float(0x7f800000), hi = -lo;
    for (int c = c_lo; c < c_hi; ++c) {
        const float d = cull[((size_t)ty * vp.tiles_x + c) * vp.K + rank];
        lo = fminf(lo, d);
        hi = fmaxf(hi, d);
    }
    chunk[i] = make_float2(lo, hi);
}

// Run boundaries of the sorted keys: a thread takes 4 consecutive keys per round (one
// 16-byte load when `vec`) and their right neighbour; grid-stride over a resident grid.
__global__ void __launch_bounds__(256)
ranges_kernel(const uint32_t* __restrict__ keys, int64_t n, bool vec, uint2* __restrict__ ranges, uint32_t first) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
    for (int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; j0 < n; j0 += stride) {
        uint32_t k[5];
        if (vec && j0 + 4 <= n) {
            const uint4 v = *reinterpret_cast<const uint4*>(keys + j0);
            k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
        } else {
            for (int q = 0; q < 4; ++q) k[q] = j0 + q < n ? keys[j0 + q] : 0u;
        }
        k[4] = j0 + 4 < n ? keys[j0 + 4] : 0u;
        const uint32_t prev = j0 > 0 ? keys[j0 - 1] : 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t j = j0 + q;
            if (j >= n) break;
            if (j == 0 || (q == 0 ? prev : k[q - 1]) != k[q]) ranges[k[q]].x = first + (uint32_t)j;
            if (j == n - 1 || k[q + 1] != k[q]) ranges[k[q]].y = first + (uint32_t)(j + 1);
        }
    }
}

// base_dev (nullable): the keys start at that index of the instance array (device value).
__global__ void ranges_dev_kernel(const uint32_t* __restrict__ keys, const unsigned long long* __restrict__ n_dev,
                                  int64_t cap, uint2* __restrict__ ranges,
                                  const unsigned long long* __restrict__ base_dev) {
    const unsigned long long nv = *n_dev;
    const int64_t n = nv < (unsigned long long)cap ? (int64_t)nv : cap;
    const uint32_t base = base_dev ? (uint32_t)*base_dev : 0u;
    keys += base;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[j];
        if (j == 0 || keys[j - 1] != k) ranges[k].x = base + (uint32_t)j;
        if (j == n - 1 || keys[j + 1] != k) ranges[k].y = base + (uint32_t)(j + 1);
    }
}

// ------------------------------------------------------------------ shared pieces of the blend
// The current subset's leaf constraints (Eq. 6) live in shared memory (LeafPath): they
// are uniform across the CTA and only read for splats held by several subsets.

// The leaf's planes that cut a tile for one staged splat, as affine tests of the pixel
// centre: float4(A, B, C, side) with side +1 (need A X + B Y + C >= 0) or -1 (need < 0).
constexpr int kMaxCutPlanes = 3;
constexpr uint32_t kPlanesAll = 7;   // more cut planes than stored: test every plane per pair

// Classifies the leaf's planes for a splat at depth z over the tile's pixel centres
// [X0, X0+15] x [Y0, Y0+15]: a plane every centre passes (with a margin far above fp32
// rounding) is dropped, one every centre fails culls the record (-1), the others are
// stored.  Returns the number stored, or kPlanesAll.
__device__ __forceinline__ int classify_planes(const ViewParams& vp, const LeafPath& lp, float z, float X0, float Y0,
                                               float4* out) {
    int n = 0;
    for (int d = 0; d < vp.L; ++d) {
        const int ar = lp.axis_right[d];
        const int a = ar & 3;
        const bool right = (ar >> 2) != 0;
        const float4 P = plane_coeffs(vp, a, lp.split[d], z);
        const float ax0 = P.x * X0, ax1 = P.x * (X0 + 15.f), by0 = P.y * Y0, by1 = P.y * (Y0 + 15.f);
        const float vmin = P.z + fminf(ax0, ax1) + fminf(by0, by1);
        const float vmax = P.z + fmaxf(ax0, ax1) + fmaxf(by0, by1);
        const float oa = a == 0 ? vp.o[0] : (a == 1 ? vp.o[1] : vp.o[2]);
        const float m = 1e-5f * (fabsf(oa) + fabsf(lp.split[d]) + 4.f * z) + 1e-6f;
        const bool pass_all = right ? vmin >= m : vmax <= -m;
        const bool fail_all = right ? vmax <= -m : vmin >= m;
        if (fail_all) return -1;
        if (pass_all) continue;
        if (n < kMaxCutPlanes) out[n] = make_float4(P.x, P.y, P.z, right ? 1.f : -1.f);
        ++n;
    }
    return n <= kMaxCutPlanes ? n : (int)kPlanesAll;
}

// Eq. 6 for one pixel: the stored cut planes, or (rarely) every plane of the leaf.
__device__ __forceinline__ bool in_subset(const float4* planes, int n, const ViewParams& vp, const LeafPath& lp,
                                          float z, float X, float Y) {
    bool ok = true;
    if (n != (int)kPlanesAll) {
        for (int c = 0; c < n; ++c) {
            const float4 P = planes[c];
            const float v = fmaf(P.x, X, fmaf(P.y, Y, P.z));
            ok = ok && (P.w > 0.f ? v >= 0.f : v < 0.f);
        }
    } else {
        for (int d = 0; d < vp.L; ++d) {
            const int ar = lp.axis_right[d];
            const float4 P = plane_coeffs(vp, ar & 3, lp.split[d], z);
            const float v = fmaf(P.x, X, fmaf(P.y, Y, P.z));
            ok = ok && ((ar >> 2) ? v >= 0.f : v < 0.f);
        }
    }
    return ok;
}

// Each warp owns an 8x4 block of the 16x16 tile: warp w covers columns 8 (w & 1) .. +7
// and rows 4 (w >> 1) .. +3, so a splat that misses a block costs that warp nothing.
__device__ __forceinline__ void thread_pixel(int tid, int& lx, int& ly) {
    const int w = tid >> 5, l = tid & 31;
    lx = ((w & 1) << 3) | (l & 7);
    ly = ((w >> 1) << 2) | (l >> 3);
}

// Tile-relative record in shared memory (3 x float4):
//   a = (mx, my, l11, l12)    centre relative to the tile origin, conic factor L = [[l11, l12], [0, l22]]
//   b = (l22, alpha, d2max, rho2)
//        d2max = min(trunc_mult^2, 2 ln(alpha / alpha_min)): a pixel passes the Mahalanobis
//        test (d2 <= trunc_mult^2) and the opacity test (alpha exp(-d2/2) >= alpha_min) iff
//        d2 <= d2max;  rho2 = (D/z)^2 of the ball test, +inf when the ball holds the whole
//        ellipse d2 <= d2max (the test cannot fail), negated when the splat straddles
//        subsets (the Eq. 6 test is needed)
//   c = (r, g, b, z)
struct StagedRec {
    float4 a;
    float4 b;
    float4 c;
};

constexpr float kInfF = __builtin_huge_valf();

// Bit w set: the footprint can touch warp w's 8x4 block (one span per 4-row band); for a
// splat held by several subsets the span is also clipped to the current subset (Eq. 6).
__device__ __forceinline__ uint32_t block_mask(const StagedRec& r, const ViewParams& vp, const LeafPath& lp, float x0t,
                                               float y0t) {
    const Footprint f = make_footprint(r.a.x, r.a.y, r.a.z, r.a.w, r.b.x, r.b.y, r.b.w, vp);
    const bool straddles = r.b.w < 0.f;
    SubsetClip clip;
    if (straddles) make_clip(vp, lp, vp.L, r.c.w, clip);
    uint32_t m = 0;
#pragma unroll
    for (int band = 0; band < 4; ++band) {
        float x0, x1;
        const float ylo = (float)(4 * band) + 0.5f - f.cy, yhi = (float)(4 * band) + 3.5f - f.cy;
        if (!footprint_span(f, vp, ylo, yhi, x0, x1)) continue;
        float X0 = f.cx + x0 + x0t, X1 = f.cx + x1 + x0t;          // absolute pixel-centre X
        if (straddles && !clip_span(clip, ylo + f.cy + y0t, yhi + f.cy + y0t, X0, X1)) continue;
        const float pl = ceilf(X0 - x0t - 0.5f), ph = floorf(X1 - x0t - 0.5f);   // tile pixel columns
        if (pl <= 7.f && ph >= 0.f) m |= 1u << (2 * band);
        if (pl <= 15.f && ph >= 8.f) m |= 1u << (2 * band + 1);
    }
    return m;
}

// True when the ball test's screen ellipse (dx/fx)^2 + (dy/fy)^2 <= rho2 holds the splat's
// ellipse d2 <= d2max, with 0.1% to spare: the largest value of (dx/fx)^2 + (dy/fy)^2 over
// the splat's ellipse is d2max times the largest eigenvalue of S Sigma' S, S = diag(1/fx, 1/fy).
__device__ __forceinline__ bool ball_holds_ellipse(const StagedRec& r, const ViewParams& vp) {
    const float l11 = r.a.z, l12 = r.a.w, l22 = r.b.x;
    const float qa = l11 * l11, qb = l11 * l12, qc = fmaf(l12, l12, l22 * l22);
    const float sd = l11 * l22, idet = 1.f / (sd * sd);
    const float mxx = qc * idet * vp.ifx * vp.ifx, myy = qa * idet * vp.ify * vp.ify;
    const float mxy = -qb * idet * vp.ifx * vp.ify;
    const float h = 0.5f * (mxx + myy), dd = 0.5f * (mxx - myy);
    const float lmax = h + sqrtf(fmaf(dd, dd, mxy * mxy));
    return fmaxf(r.b.z, 0.f) * lmax * 1.001f + 1e-30f <= fabsf(r.b.w);
}

__device__ __forceinline__ StagedRec stage_record(const float4* __restrict__ rec, uint32_t id, float x0, float y0,
                                                  const ViewParams& vp) {
    const float4 r0 = rec[3 * (size_t)id], r1 = rec[3 * (size_t)id + 1], r2 = rec[3 * (size_t)id + 2];
    uint32_t lo_bits = __float_as_uint(r0.z);
    __half2 lo = *reinterpret_cast<__half2*>(&lo_bits);
    float2 lof = __half22float2(lo);
    StagedRec s;
    s.a = make_float4(__fadd_rn(__fsub_rn(r0.x, x0), lof.x), __fadd_rn(__fsub_rn(r0.y, y0), lof.y), r1.x, r1.y);
    const float d2max = fminf(vp.trunc_mult * vp.trunc_mult, 2.f * logf(r0.w / vp.alpha_min));
    s.b = make_float4(r1.z, r0.w, d2max, r1.w);
    s.c = make_float4(r2.x, r2.y, r2.z, r2.w);
    return s;
}

// Stages record `id` for the current subset (the whole block calls it, one record per
// thread): its tile-relative form, the mask of warp blocks it can touch, and for a
// straddling splat the leaf planes that cut the tile (stored in `planes`; their count in
// mask bits 8-10).  A mask of 0 drops the record.
__device__ __forceinline__ void stage_for_subset(const float4* __restrict__ rec, uint32_t id, float x0, float y0,
                                                 const ViewParams& vp, const LeafPath& lp, StagedRec& sr,
                                                 uint32_t& msk, float4* planes) {
    sr = stage_record(rec, id, x0, y0, vp);
    msk = sr.b.z >= 0.f ? block_mask(sr, vp, lp, x0, y0) : 0u;
    if (sr.b.w < 0.f && msk) {
        const int nc = classify_planes(vp, lp, sr.c.w, x0 + 0.5f, y0 + 0.5f, planes);
        if (nc < 0) msk = 0;                        // no pixel of the tile is in this subset
        else if (nc == 0) sr.b.w = -sr.b.w;         // every pixel is: no per-pixel test
        else msk |= (uint32_t)nc << 8;
    }
    if (msk && ball_holds_ellipse(sr, vp)) sr.b.w = copysignf(kInfF, sr.b.w);
    // rho2 = +inf marks the records whose pairs need only the Mahalanobis test: the ball
    // holds the ellipse, one subset holds every pixel, and alpha < alpha_max (so that
    // sigma = alpha G needs no clamp); a record whose ball holds the ellipse but whose
    // alpha reaches alpha_max keeps a ball bound that never fails instead
    if (sr.b.w == kInfF && !(sr.b.y < vp.alpha_max)) sr.b.w = __int_as_float(0x7f7fffff);
}

// Compacts, per warp, the staged records whose mask has the warp's bit: wl[0..n) in
// record order.  Returns n (uniform across the warp).
// kHoist: all eight mask loads issued before the first ballot (faster in the forward; the
// backward, with more live registers, keeps the loop).
template <bool kHoist>
__device__ __forceinline__ int warp_list(const uint32_t* smask, int nb, int warp, int lane, uint8_t* wl) {
    int n = 0;
    const unsigned lower = (1u << lane) - 1u;
    if (kHoist) {
        uint32_t m[kBlendThreads / 32];
#pragma unroll
        for (int c = 0; c < kBlendThreads / 32; ++c) m[c] = smask[c * 32 + lane];
#pragma unroll
        for (int c = 0; c < kBlendThreads / 32; ++c) {
            const bool hit = c * 32 + lane < nb && ((m[c] >> warp) & 1u);
            const unsigned bits = __ballot_sync(0xffffffffu, hit);
            if (hit) wl[n + __popc(bits & lower)] = (uint8_t)(c * 32 + lane);
            n += __popc(bits);
        }
    } else {
        for (int c0 = 0; c0 < nb; c0 += 32) {
            const bool hit = c0 + lane < nb && ((smask[c0 + lane] >> warp) & 1u);
            const unsigned bits = __ballot_sync(0xffffffffu, hit);
            if (hit) wl[n + __popc(bits & lower)] = (uint8_t)(c0 + lane);
            n += __popc(bits);
        }
    }
    __syncwarp();
    return n;
}

// The truncation tests of one (pixel, record) pair (Sec. 3.1 and Eq. 6): d2 <= d2max, the
// ball test unless the ball holds the ellipse, and the subset test for straddling splats.
// Identical in the forward and the backward, so both take the same decisions.
__device__ __forceinline__ bool pair_passes(const float4& B, const float4& Cc, float dx, float dy, float d2,
                                            const float4* planes, uint32_t msk, const ViewParams& vp,
                                            const LeafPath& lp, float Xc, float Yc) {
    // the ball test without a branch: |rho2| is +inf when the ball holds the ellipse
    const float bx = dx * vp.ifx, by = dy * vp.ify;
    bool ok = (d2 <= B.z) & (fmaf(bx, bx, by * by) <= fabsf(B.w));
    if (B.w < 0.f) ok = ok && in_subset(planes, (int)((msk >> 8) & 7u), vp, lp, Cc.w, Xc, Yc);   // warp-uniform
    return ok;
}

// warp-aggregated pair counters (tracing only)
__device__ __forceinline__ void count_add(unsigned long long* dst, uint32_t v) {
    unsigned long long e = v;
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0 && e) atomicAdd(dst, e);
}

__device__ __forceinline__ void count_pairs(unsigned long long* pairs, uint32_t n_eval, uint32_t n_contrib) {
    unsigned long long e = n_eval, c = n_contrib;
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(pairs, e);
        atomicAdd(pairs + 1, c);
    }
}

// ------------------------------------------------------------------ blend forward
// Termination: a pixel whose transmittance is below eps_T at the start of a group of 32
// entries of its warp's record list is frozen for the rest of the subset (T is kept and
// set to 0, so later pairs add nothing); the check happens per group only, so the
// per-pair loop carries no termination logic.  The backward freezes at the same points.
//
// One tile of the view: `ranges` and `tile_depth` point at the tile's K entries (view
// rank order); pC/pT (partial maps) and tile_depth may be null.  The whole block calls it.
//
// ends (nullable, the tile's K ranges again): where a subset saturated the tile, the
// range's end is moved back to the end of the last batch staged, so that a backward
// replaying these lists stops where the forward did.
//
// Groups of ranks (the image-only forward binned group by group): the call blends view
// ranks [r_begin, r_end) only.  With r_begin > 0 each pixel's merged colour and
// transmittance in front come from `state` (a float4 per pixel, 256 per tile); with
// r_end < K a tile that still has a pixel whose front transmittance is at least eps_T
// stores them there and sets its flag in `open`, and a tile with none writes its image
// (nothing behind can change it), clears its flag and marks the later ranks' depths -inf.
template <bool kCount>
__device__ __forceinline__ void blend_fwd_tile(const ViewParams& vp, const TreeParams& tp, int tile,
                                               const uint2* ranges, const uint32_t* __restrict__ ival,
                                               const float4* __restrict__ rec, float* __restrict__ pC,
                                               float* __restrict__ pT, float* __restrict__ image,
                                               float* __restrict__ Tfin, float* __restrict__ tile_depth,
                                               uint2* ends, unsigned long long* __restrict__ pairs,
                                               int r_begin = 0, int r_end = -1, float4* __restrict__ state = nullptr,
                                               uint8_t* __restrict__ open = nullptr) {
    if (r_end < 0) r_end = vp.K;
    __shared__ StagedRec srec[kBlendThreads];
    __shared__ uint32_t smask[kBlendThreads];
    __shared__ float4 splane[kBlendThreads][kMaxCutPlanes];
    __shared__ uint8_t wlist[kBlendThreads / 32][kBlendThreads];
    __shared__ LeafPath lp;
    __shared__ uint32_t sused[kBlendThreads];
    // per-pixel values touched once per subset live in shared memory (register budget)
    __shared__ float s_img[4][kBlendThreads];   // merged colour so far and the transmittance in front
    __shared__ float s_tkeep[kBlendThreads];    // T of a frozen pixel
    uint32_t n_eval = 0, n_contrib = 0, n_d2 = 0, n_ball = 0, n_leaf = 0, n_strad = 0, n_staged = 0, n_used = 0;
    uint32_t n_iter = 0;   // warp passes over one list entry (lane 0 counts)
    uint32_t n_behind = 0; // pairs evaluated where the merged front transmittance is below eps_T
    const int tyi = tile / vp.tiles_x, txi = tile - tyi * vp.tiles_x;
    int lx, ly;
    thread_pixel(threadIdx.x, lx, ly);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px = txi * kTile + lx, py = tyi * kTile + ly;
    const bool inside = px < vp.W && py < vp.H;
    const float x0 = (float)(txi * kTile), y0 = (float)(tyi * kTile);
    const float pcx = lx + 0.5f, pcy = ly + 0.5f;
    const size_t HW = (size_t)vp.W * vp.H;
    const size_t pix = (size_t)py * vp.W + px;
    uint8_t* wl = wlist[warp];
    const int tid = threadIdx.x;
    if (r_begin > 0 && inside) {
        const float4 st = state[(size_t)tile * kBlendThreads + threadIdx.x];
        s_img[0][tid] = st.x;
        s_img[1][tid] = st.y;
        s_img[2][tid] = st.z;
        s_img[3][tid] = st.w;
    } else {
        s_img[0][tid] = 0.f;
        s_img[1][tid] = 0.f;
        s_img[2][tid] = 0.f;
        s_img[3][tid] = 1.f;
    }

    // Culling (always without partial maps, where only the image is wanted; with them when
    // the options ask for it): a pixel whose transmittance in front of subset k (the merge's
    // P) is below eps_T skips k and every later subset (they change its colour by less than
    // eps_T max(rgb); its partials there stay C = 0, T = 1), and a tile with no pixel left
    // skips the subset.
    const bool cull = pC == nullptr || vp.cull_occluded != 0;
    for (int r = r_begin; r < r_end; ++r) {
        const int k = vp.order[r];
        const uint2 rg = ranges[r];
        const bool live = inside && !(cull && s_img[3][tid] < vp.eps_T);
        if (cull && __syncthreads_count(live) == 0) {
            if (tile_depth && threadIdx.x == 0) tile_depth[r] = -kInfF;   // nothing blended, nothing needed
            if (ends && threadIdx.x == 0) ends[r].y = rg.x;                 // nothing for a backward to replay
            if (inside && pC) {
                pC[((size_t)k * 3 + 0) * HW + pix] = 0.f;
                pC[((size_t)k * 3 + 1) * HW + pix] = 0.f;
                pC[((size_t)k * 3 + 2) * HW + pix] = 0.f;
                pT[(size_t)k * HW + pix] = 1.f;
            }
            continue;
        }
        if (threadIdx.x == 0) leaf_path(tp, k, lp);   // read only after the next barrier
        float C0 = 0.f, C1 = 0.f, C2 = 0.f;
        float T = live ? 1.f : 0.f;
        bool frozen = !live;
        float zsat = kInfF;   // the subset never saturated the tile
        uint32_t send = rg.y;  // end of the last batch staged
        const bool behind_front = kCount && s_img[3][tid] < vp.eps_T;
        for (uint32_t b0 = rg.x; b0 < rg.y; b0 += kBlendThreads) {
            const int nb = (int)min((uint32_t)kBlendThreads, rg.y - b0);
            __syncthreads();
            if ((int)threadIdx.x < nb) {
                StagedRec sr;
                uint32_t msk;
                stage_for_subset(rec, ival[b0 + threadIdx.x], x0, y0, vp, lp, sr, msk, splane[threadIdx.x]);
                srec[threadIdx.x] = sr;
                smask[threadIdx.x] = msk;
                if (kCount) {
                    sused[threadIdx.x] = 0;
                    ++n_staged;
                }
            }
            __syncthreads();
            const int n = warp_list<true>(smask, nb, warp, lane, wl);
            for (int t0 = 0; t0 < n; t0 += 32) {
                if (!frozen && T < vp.eps_T) {
                    frozen = true;
                    s_tkeep[tid] = T;
                    T = 0.f;
                }
                if (__all_sync(0xffffffffu, frozen)) break;
                const int t1 = min(n, t0 + 32);
                // a group of simple records only (the Mahalanobis test alone, no clamp) takes
                // the same arithmetic with no per-pair branch
                bool all_simple = false;
                if (!kCount) {
                    const bool simple_l = t0 + lane >= t1 || srec[wl[t0 + lane]].b.w == kInfF;
                    all_simple = __all_sync(0xffffffffu, simple_l);
                }
                if (all_simple) {
                    #pragma unroll 2
                    for (int t = t0; t < t1; ++t) {
                        const int j = wl[t];
                        const float4 A = srec[j].a;
                        const float4 B = srec[j].b;
                        const float4 Cc = srec[j].c;
                        const float dx = pcx - A.x, dy = pcy - A.y;
                        const float u1 = fmaf(A.z, dx, A.w * dy), u2 = B.x * dy;
                        const float d2 = fmaf(u1, u1, u2 * u2);
                        const float G = ex2_approx(d2 * kNegHalfLog2e);
                        const float sig = d2 <= B.z ? B.y * G : 0.f;
                        const float w = sig * T;
                        C0 = fmaf(Cc.x, w, C0);
                        C1 = fmaf(Cc.y, w, C1);
                        C2 = fmaf(Cc.z, w, C2);
                        T = fmaf(-sig, T, T);
                    }
                    continue;
                }
                #pragma unroll 2
                for (int t = t0; t < t1; ++t) {
                    if (kCount && lane == 0) ++n_iter;
                    const int j = wl[t];
                    const float4 A = srec[j].a;
                    const float4 B = srec[j].b;
                    const float4 Cc = srec[j].c;
                    const float dx = pcx - A.x, dy = pcy - A.y;
                    const float u1 = fmaf(A.z, dx, A.w * dy), u2 = B.x * dy;
                    const float d2 = fmaf(u1, u1, u2 * u2);
                    const float G = ex2_approx(d2 * kNegHalfLog2e);
                    bool ok;
                    float sig;
                    if (B.w == kInfF) {   // warp-uniform: the Mahalanobis test alone, no clamp
                        ok = d2 <= B.z;
                        sig = ok ? B.y * G : 0.f;
                    } else {
                        ok = pair_passes(B, Cc, dx, dy, d2, splane[j], smask[j], vp, lp, x0 + pcx, y0 + pcy);
                        sig = ok ? fminf(B.y * G, vp.alpha_max) : 0.f;
                    }
                    if (kCount && !frozen) {
                        ++n_eval;
                        n_behind += behind_front;
                        n_strad += B.w < 0.f;
                        n_d2 += !(d2 <= B.z);
                        const bool in_ball = !(fabsf(B.w) != kInfF) ||
                                             fmaf(dx * vp.ifx, dx * vp.ifx, (dy * vp.ify) * (dy * vp.ify)) <= fabsf(B.w);
                        n_ball += d2 <= B.z && !in_ball;
                        n_leaf += d2 <= B.z && in_ball && !ok;
                        n_contrib += ok;
                        if (ok) sused[j] = 1;
                    }
                    const float w = sig * T;
                    C0 = fmaf(Cc.x, w, C0);
                    C1 = fmaf(Cc.y, w, C1);
                    C2 = fmaf(Cc.z, w, C2);
                    T = fmaf(-sig, T, T);
                }
            }
            if (kCount) {
                __syncthreads();
                if ((int)threadIdx.x < nb) n_used += sused[threadIdx.x];
            }
            if (__syncthreads_count(frozen || T < vp.eps_T) == kBlendThreads) {
                zsat = srec[nb - 1].c.w;   // depth of the last instance staged
                send = b0 + (uint32_t)nb;
                break;
            }
        }
        if (frozen && inside) T = live ? s_tkeep[tid] : 1.f;
        if (tile_depth && threadIdx.x == 0) tile_depth[r] = zsat;
        if (ends && threadIdx.x == 0 && send != rg.y) ends[r].y = send;
        if (inside) {
            if (pC) {
                pC[((size_t)k * 3 + 0) * HW + pix] = C0;
                pC[((size_t)k * 3 + 1) * HW + pix] = C1;
                pC[((size_t)k * 3 + 2) * HW + pix] = C2;
                pT[(size_t)k * HW + pix] = T;
            }
            const float Pm = s_img[3][tid];
            s_img[0][tid] = fmaf(C0, Pm, s_img[0][tid]);
            s_img[1][tid] = fmaf(C1, Pm, s_img[1][tid]);
            s_img[2][tid] = fmaf(C2, Pm, s_img[2][tid]);
            s_img[3][tid] = Pm * T;
        }
    }
    if (r_end < vp.K) {
        // end of a group: keep the state of a tile that later ranks can still change
        const bool open_px = inside && !(s_img[3][tid] < vp.eps_T);
        if (__syncthreads_count(open_px) > 0) {
            if (inside)
                state[(size_t)tile * kBlendThreads + tid] = make_float4(s_img[0][tid], s_img[1][tid], s_img[2][tid],
                                                                   s_img[3][tid]);
            if (tid == 0) open[tile] = 1;
            image = nullptr;   // the last group writes it
        } else {
            if (tid == 0) open[tile] = 0;
            if (tile_depth && tid < vp.K && tid >= r_end) tile_depth[tid] = -kInfF;   // nothing needed behind
        }
    }
    if (inside && image) {
        const float Pm = s_img[3][tid];
        image[0 * HW + pix] = fmaf(vp.bg[0], Pm, s_img[0][tid]);
        image[1 * HW + pix] = fmaf(vp.bg[1], Pm, s_img[1][tid]);
        image[2 * HW + pix] = fmaf(vp.bg[2], Pm, s_img[2][tid]);
        if (Tfin) Tfin[pix] = Pm;
    }
    if (kCount) {
        count_pairs(pairs, n_eval, n_contrib);
        count_add(pairs + 4, n_d2);
        count_add(pairs + 5, n_ball);
        count_add(pairs + 6, n_leaf);
        count_add(pairs + 7, n_strad);
        count_add(pairs + 8, n_staged);
        count_add(pairs + 10, n_iter);
        count_add(pairs + 9, n_used);
        count_add(pairs + 11, n_behind);
    }
}

template <bool kCount>
__global__ void __launch_bounds__(kBlendThreads, RGS_BLEND_MIN_BLOCKS)
blend_fwd_kernel(ViewParams vp, TreeParams tp, uint2* ranges, const uint32_t* __restrict__ ival,
                 const float4* __restrict__ rec, float* __restrict__ pC, float* __restrict__ pT,
                 float* __restrict__ image, float* __restrict__ Tfin, float* __restrict__ tile_depth, bool record_ends,
                 unsigned long long* __restrict__ pairs, int r_begin, int r_end, float4* __restrict__ state,
                 uint8_t* __restrict__ open, const unsigned long long* __restrict__ skip) {
    if (skip && *skip) return;   // a batch's overflow flag, or an unused request slot
    const int tile = blockIdx.x;
    if (r_begin > 0 && !open[tile]) return;   // closed by an earlier group (uniform across the block)
    uint2* tr = ranges + (size_t)tile * vp.K;
    blend_fwd_tile<kCount>(vp, tp, tile, tr, ival, rec, pC, pT, image, Tfin,
                           tile_depth ? tile_depth + (size_t)tile * vp.K : nullptr, record_ends ? tr : nullptr, pairs,
                           r_begin, r_end, state, open);
}

// Persistent forward blend over the global tiles of a batch: each block takes the next
// tile from a device counter until all are done; a tile belongs to the last request
// whose tile_base it reaches.  The request's view is kept in shared memory while
// consecutive tiles stay in one request.
__global__ void __launch_bounds__(kBlendThreads, RGS_BLEND_MIN_BLOCKS)
blend_batch_kernel(const BatchSlot* __restrict__ slots, const BatchHeader* __restrict__ hdr, TreeParams tp,
                   uint2* __restrict__ ranges, const uint32_t* __restrict__ ival, const float4* __restrict__ rec,
                   unsigned long long* __restrict__ counters, bool record_ends) {
    __shared__ ViewParams svp;
    __shared__ uint32_t s_tile;
    __shared__ int s_slot;
    if (counters[2]) return;   // overflow: the batch is discarded
    const int S = hdr->S;
    const uint32_t total = hdr->total_tiles;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t t = (uint32_t)atomicAdd(&counters[3], 1ull);
            int sl = 0;
            while (sl + 1 < S && hdr->tile_base[sl + 1] <= t) ++sl;
            s_tile = t;
            s_slot = sl;
        }
        __syncthreads();
        const uint32_t t = s_tile;
        const int slot = s_slot;
        if (t >= total) break;
        if (slot != cur) {
            constexpr int kWords = (int)(sizeof(ViewParams) / 4);
            for (int w = threadIdx.x; w < kWords; w += blockDim.x)
                reinterpret_cast<uint32_t*>(&svp)[w] = reinterpret_cast<const uint32_t*>(&slots[slot].vp)[w];
            cur = slot;
            __syncthreads();
        }
        uint2* tr = ranges + (size_t)t * svp.K;
        blend_fwd_tile<false>(svp, tp, (int)(t - hdr->tile_base[slot]), tr, ival, rec, nullptr, nullptr,
                              slots[slot].image, nullptr, nullptr, record_ends ? tr : nullptr, nullptr);
        __syncthreads();   // s_tile is rewritten by the next claim
    }
}

// ------------------------------------------------------------------ foot reading (forward only)
// Under the comparison reading of Sec. 3.2, x_i is the foot of the perpendicular from the
// centre onto the pixel ray, and a ray's contributors are ordered by the foot's ray
// parameter t.  For pixel centre (X, Y) and a splat at depth z with projected centre
// (mx, my), with a = X - cx, c = Y - cy, b = mx - cx, d = my - cy and k = fx^2 / fy^2,
//   s(p) = fx^2 |r_p| t = z (fx^2 + a b + k c d),       r_p = (a / fx, c / fy, 1),
// an order key free of the roundings of 1/fx (a, c and fx^2 + ... are nearly exact), so
// that the fp32 key errs by about 1e-7 of its size.  The order changes from pixel to
// pixel.  The instances of a (tile, subset) run are sorted by a lower bound of s over the
// tile; each pixel keeps the contributors it has accepted in a small buffer ordered by s
// and blends one only when the next instance's bound shows that nothing later can come
// before it.  Exact unless the buffer overflows (counted); then its nearest entry is
// blended early.
constexpr int kFootPend = 64;   // pending contributors per pixel (power of two)

// fx^2 and k = fx^2 / fy^2 of the key, rounded the same way wherever they are used.
__device__ __forceinline__ float2 foot_scale(const ViewParams& vp) {
    const float fx2 = __fmul_rn(vp.fx, vp.fx);
    return make_float2(fx2, __fdiv_rn(fx2, __fmul_rn(vp.fy, vp.fy)));
}

// Lower bound of s over the pixel centres [px0, px1] x [py0, py1] for a splat with
// projected centre (mx, my) at depth z, less a margin (1e-5 of the size of its terms) far
// above the fp32 error of the per-pixel s.
__device__ __forceinline__ float foot_bound_px(float mx, float my, float z, int px0, int px1, int py0, int py1,
                                               const ViewParams& vp) {
    const float2 sc = foot_scale(vp);
    const float b = __fsub_rn(mx, vp.cx), d = __fsub_rn(my, vp.cy);
    const float a0 = __fsub_rn((float)px0 + 0.5f, vp.cx), a1 = __fsub_rn((float)px1 + 0.5f, vp.cx);
    const float c0 = __fmul_rn(__fsub_rn((float)py0 + 0.5f, vp.cy), sc.y);
    const float c1 = __fmul_rn(__fsub_rn((float)py1 + 0.5f, vp.cy), sc.y);
    const float ax = fminf(__fmul_rn(a0, b), __fmul_rn(a1, b));
    const float ay = fminf(__fmul_rn(c0, d), __fmul_rn(c1, d));
    const float q = __fadd_rn(__fadd_rn(sc.x, ax), ay);
    const float size = __fmul_rn(z, __fadd_rn(__fadd_rn(sc.x, fabsf(ax)), fabsf(ay)));
    return __fsub_rn(__fmul_rn(z, q), __fmul_rn(size, 1e-5f));
}

// The bound over the pixels of tile (tx, ty) inside the image: the sort key of an
// instance.  The key kernel and the blend evaluate it on the same record values with
// explicit roundings, so the blend sees the bounds the sort used.
__device__ __forceinline__ float foot_bound(float mx, float my, float z, int tx, int ty, const ViewParams& vp) {
    return foot_bound_px(mx, my, z, tx * kTile, min(tx * kTile + kTile - 1, vp.W - 1), ty * kTile,
                         min(ty * kTile + kTile - 1, vp.H - 1), vp);
}

// Warp blocks of the tile that a staged record can touch under the foot reading: per
// 4-row band the footprint's span, clipped for a straddling splat to subset k over the
// foot's depth range in that band (the count's and emission's rule at band resolution).
__device__ __forceinline__ uint32_t foot_block_mask(const StagedRec& r, const ViewParams& vp, int k, float zr,
                                                    float x0t, float y0t) {
    Footprint f = make_footprint(r.a.x, r.a.y, r.a.z, r.a.w, r.b.x, r.b.y, fabsf(r.b.w), vp);
    f.zr = zr;
    const bool straddles = r.b.w < 0.f;
    uint32_t m = 0;
#pragma unroll
    for (int band = 0; band < 4; ++band) {
        float x0, x1;
        const float ylo = (float)(4 * band) + 0.5f - f.cy, yhi = (float)(4 * band) + 3.5f - f.cy;
        if (!footprint_span(f, vp, ylo, yhi, x0, x1)) continue;
        float X0 = f.cx + x0 + x0t, X1 = f.cx + x1 + x0t;          // absolute pixel-centre X
        if (straddles) {
            const float Ylo = ylo + f.cy + y0t, Yhi = yhi + f.cy + y0t;
            Footprint fa = f;   // absolute centre for the depth range
            fa.cx = f.cx + x0t;
            fa.cy = f.cy + y0t;
            float za, zb;
            if (foot_depth_range(fa, vp, r.c.w, fmaxf(X0, x0t + 0.5f), fminf(X1, x0t + 15.5f), Ylo, Yhi, za, zb) &&
                !clip_span_depths(vp, k, vp.L, za, zb, Ylo, Yhi, X0, X1))
                continue;
        }
        const float pl = ceilf(X0 - x0t - 0.5f), ph = floorf(X1 - x0t - 0.5f);   // tile pixel columns
        if (pl <= 7.f && ph >= 0.f) m |= 1u << (2 * band);
        if (pl <= 15.f && ph >= 8.f) m |= 1u << (2 * band + 1);
    }
    return m;
}

// Float bits mapped so that unsigned order is float order (negative bounds included).
__device__ __forceinline__ uint32_t ordered_bits(float v) {
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Per instance: the bound of its (splat, tile) and its position, for the first sort pass.
__global__ void foot_keys_kernel(ViewParams vp, const uint32_t* __restrict__ ikey, const uint32_t* __restrict__ ival,
                                 int64_t n, const float4* __restrict__ rec, uint32_t* __restrict__ fkey,
                                 uint32_t* __restrict__ fidx) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t tile = ikey[i] >> vp.L;
        const int ty = (int)(tile / (uint32_t)vp.tiles_x), tx = (int)(tile - (uint32_t)ty * vp.tiles_x);
        const uint32_t id = ival[i];
        const float4 r0 = rec[3 * (size_t)id];
        const float z = rec[3 * (size_t)id + 2].w;
        fkey[i] = ordered_bits(foot_bound(r0.x, r0.y, z, tx, ty, vp));
        fidx[i] = (uint32_t)i;
    }
}

// (tile, subset) keys and payloads in the order of the bound sort.
__global__ void foot_gather_kernel(const uint32_t* __restrict__ idx, int64_t n, const uint32_t* __restrict__ ikey,
                                   const uint32_t* __restrict__ ival, uint32_t* __restrict__ k2,
                                   uint32_t* __restrict__ v2) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = idx[j];
        k2[j] = ikey[i];
        v2[j] = ival[i];
    }
}

// Eq. 6 at the foot: x = o + zf R^T r_p, with zf = s / (fx^2 |r_p|^2) the foot's camera
// depth and g = R^T r_p; right of a node iff x[a] >= split (the half-open rule).  Every leaf
// tests a node with the same arithmetic, so the decisions of two leaves are complementary.
__device__ __forceinline__ bool in_subset_foot(const LeafPath& lp, int L, float zf, float g0, float g1, float g2,
                                               const ViewParams& vp) {
    bool ok = true;
#pragma unroll
    for (int d = 0; d < kMaxRenderDepth; ++d) {
        if (d >= L) break;
        const int ar = lp.axis_right[d];
        const int a = ar & 3;
        const float ga = a == 0 ? g0 : (a == 1 ? g1 : g2);
        const float oa = a == 0 ? vp.o[0] : (a == 1 ? vp.o[1] : vp.o[2]);
        const float xa = fmaf(zf, ga, oa);
        ok = ok && ((ar >> 2) ? (xa >= lp.split[d]) : (xa < lp.split[d]));
    }
    return ok;
}

// One pixel's pending contributors: a ring of kFootPend entries in ascending key (the
// float pair s + sl, equal keys in arrival order) starting at `head`, `n` of them; head,
// n and the head's s (`hs`, +inf when empty) stay in registers.  An entry keeps the splat
// id, and its colour is read back from the record when it is blended.
struct FootPending {
    float s[kFootPend], sl[kFootPend], sig[kFootPend];
    uint32_t id[kFootPend];
};

__device__ __forceinline__ void foot_pop(FootPending& P, const float4* __restrict__ rec, int& head, int& n, float& hs,
                                         float& C0, float& C1, float& C2, float& T) {
    const int q = head;
    const float4 c = rec[3 * (size_t)P.id[q] + 2];
    const float w = P.sig[q] * T;
    C0 = fmaf(c.x, w, C0);
    C1 = fmaf(c.y, w, C1);
    C2 = fmaf(c.z, w, C2);
    T = fmaf(-P.sig[q], T, T);
    head = (q + 1) & (kFootPend - 1);
    --n;
    hs = n > 0 ? P.s[head] : kInfF;
}

__device__ __forceinline__ void foot_insert(FootPending& P, const float4* __restrict__ rec, int& head, int& n,
                                            float& hs, float s, float sl, float sig, uint32_t id, float& C0,
                                            float& C1, float& C2, float& T, uint32_t& n_over) {
    if (n == kFootPend) {
        foot_pop(P, rec, head, n, hs, C0, C1, C2, T);
        ++n_over;
    }
    int i = n;
    while (i > 0) {
        const int prev = (head + i - 1) & (kFootPend - 1);
        if (P.s[prev] < s || (P.s[prev] == s && P.sl[prev] <= sl)) break;
        const int to = (head + i) & (kFootPend - 1);
        P.s[to] = P.s[prev];
        P.sl[to] = P.sl[prev];
        P.sig[to] = P.sig[prev];
        P.id[to] = P.id[prev];
        --i;
    }
    const int at = (head + i) & (kFootPend - 1);
    P.s[at] = s;
    P.sl[at] = sl;
    P.sig[at] = sig;
    P.id[at] = id;
    ++n;
    if (i == 0) hs = s;
}

// Adds a float4 into global memory with one vector reduction.
__device__ __forceinline__ void red_add_v4(float4* addr, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

// The adjoint of one blended pair (flat form, Eq. 2): with T the transmittance in front of
// it inside its subset, gC = dL/dC times the transmittance in front of the subset, acc the
// pixel's <gC, colour> blended so far (this pair included) and q = <dL/dC, image>,
//   h = sigma dL/dsigma = sigma (T <gC, c> - (q - acc) / (1 - sigma))   (0 when clamped),
// and the pair's 2D gradients, added to the splat's record with vector reductions:
//   mean h L^T u (u = L delta, delta = pixel centre - centre), conic -h/2 (dx^2, 2 dx dy,
//   dy^2), alpha h / alpha, colour gC sigma T.
// Used by the foot reading's backward, whose pairs are blended in a per-pixel order.
__device__ __forceinline__ void pair_adjoint_add(const float4* __restrict__ rec, uint32_t id, float sig, float T,
                                                 float4 c, float gC0, float gC1, float gC2, float q, float& acc,
                                                 float pcx, float pcy, float x0, float y0, float alpha_max,
                                                 float4* __restrict__ g2d) {
    const float w = sig * T;
    const float grgb = gC0 * c.x + gC1 * c.y + gC2 * c.z;
    acc = fmaf(w, grgb, acc);
    const float dsig = T * grgb - __fdividef(q - acc, 1.f - sig);
    const float h = sig < alpha_max ? sig * dsig : 0.f;
    const float4 r0 = rec[3 * (size_t)id], r1 = rec[3 * (size_t)id + 1];
    uint32_t lo_bits = __float_as_uint(r0.z);
    const float2 lof = __half22float2(*reinterpret_cast<__half2*>(&lo_bits));
    const float dx = pcx - __fadd_rn(__fsub_rn(r0.x, x0), lof.x), dy = pcy - __fadd_rn(__fsub_rn(r0.y, y0), lof.y);
    const float u1 = fmaf(r1.x, dx, r1.y * dy), u2 = r1.z * dy;
    const float hdx = h * dx, hdy = h * dy;
    float4* dst = g2d + 3 * (size_t)id;
    red_add_v4(dst, make_float4(h * r1.x * u1, h * fmaf(r1.y, u1, r1.z * u2), -0.5f * hdx * dx, -hdx * dy));
    red_add_v4(dst + 1, make_float4(-0.5f * hdy * dy, __fdividef(h, r0.w), gC0 * w, gC1 * w));
    atomicAdd(&dst[2].x, gC2 * w);
}

// Blend of one tile under the foot reading: the structure of the depth-plane forward
// (subsets in view order, batches staged in shared memory, per-warp lists, freezing below
// eps_T, the merge of Eq. 5 in shared memory), with the per-pixel order restored through
// the pending buffer.  A contributor's key s = z (fx^2 + a b + k c d) is carried as a float
// pair (b = mx - cx, d = my - cy and z from the projection's float pairs; a and, for square
// pixels, k c exact), so that the order is exact to about 1e-12 of the key.  `over` counts
// buffer overflows.
//
// kBwd: the backward of that forward (flat form).  The same replay, the same pairs in the
// same per-pixel order and the same freeze points; `image` is the forward's image (read),
// gI is dL/dimage, and each blended pair adds its adjoint to g2d (pair_adjoint_add).
// Pixels with dL/dC = 0 are left out (they add nothing).  pC, pT and Tfin are unused.
template <bool kBwd>
__global__ void __launch_bounds__(kBlendThreads, 2)
blend_foot_kernel(ViewParams vp, TreeParams tp, const uint2* __restrict__ ranges_all, const uint32_t* __restrict__ ival,
                  const float4* __restrict__ rec, const float4* __restrict__ side, float* __restrict__ pC,
                  float* __restrict__ pT, float* __restrict__ image, float* __restrict__ Tfin,
                  unsigned long long* __restrict__ over, const float* __restrict__ gI, float4* __restrict__ g2d) {
    __shared__ StagedRec srec[kBlendThreads];
    __shared__ uint32_t smask[kBlendThreads];
    __shared__ float sbound[kBlendThreads];
    __shared__ float4 skey[kBlendThreads];     // (b hi, b lo, d hi, d lo)
    __shared__ float2 sextra[kBlendThreads];   // ((D/z)^2, z lo)
    __shared__ uint32_t sid[kBlendThreads];
    __shared__ float4 sctr[kBlendThreads];     // (mx, my, z, -): inputs of the warp-block bounds
    // per warp and list entry: a lower bound of s, over the warp's 8x4 block, for that
    // entry and every later one (the suffix minimum of the entries' block bounds, capped
    // by the tile bound of the batch's last record, below every later batch)
    __shared__ float wthr[kBlendThreads / 32][kBlendThreads];
    __shared__ uint8_t wlist[kBlendThreads / 32][kBlendThreads];
    __shared__ LeafPath lp;
    __shared__ float s_img[4][kBlendThreads];
    __shared__ float s_tkeep[kBlendThreads];
    const int tile = blockIdx.x;
    const uint2* ranges = ranges_all + (size_t)tile * vp.K;
    const int tyi = tile / vp.tiles_x, txi = tile - tyi * vp.tiles_x;
    int lx, ly;
    thread_pixel(threadIdx.x, lx, ly);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px = txi * kTile + lx, py = tyi * kTile + ly;
    const bool inside = px < vp.W && py < vp.H;
    const float x0 = (float)(txi * kTile), y0 = (float)(tyi * kTile);
    const float pcx = lx + 0.5f, pcy = ly + 0.5f;
    const size_t HW = (size_t)vp.W * vp.H;
    const size_t pix = (size_t)py * vp.W + px;
    const int tid = threadIdx.x;
    // per-pixel ray: a = X - cx and k c (key units), fx^2 as a float pair, r_p, |r_p|^2
    // and g = R^T r_p
    const float2 sc = foot_scale(vp);
    float Fh, Fl;
    two_prod(vp.fx, vp.fx, Fh, Fl);
    const float pa = (float)px + 0.5f - vp.cx, pc = ((float)py + 0.5f - vp.cy) * sc.y;
    const float rx = ((float)px + 0.5f - vp.cx) * vp.ifx, ry = ((float)py + 0.5f - vp.cy) * vp.ify;
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, 1.f));
    const float izf = 1.f / (sc.x * r2);   // foot depth = s / (fx^2 |r_p|^2)
    const float g0 = fmaf(vp.R[0], rx, fmaf(vp.R[3], ry, vp.R[6]));
    const float g1 = fmaf(vp.R[1], rx, fmaf(vp.R[4], ry, vp.R[7]));
    const float g2 = fmaf(vp.R[2], rx, fmaf(vp.R[5], ry, vp.R[8]));
    // backward: dL/dC of the pixel, <dL/dC, image> and <gC, colour blended so far>
    float gI0 = 0.f, gI1 = 0.f, gI2 = 0.f, qf = 0.f, acc = 0.f;
    if (kBwd && inside) {
        gI0 = gI[pix];
        gI1 = gI[HW + pix];
        gI2 = gI[2 * HW + pix];
        qf = gI0 * image[pix] + gI1 * image[HW + pix] + gI2 * image[2 * HW + pix];
    }
    const bool want = !kBwd || gI0 != 0.f || gI1 != 0.f || gI2 != 0.f;
    uint8_t* wl = wlist[warp];
    // the warp's 8x4 pixel block, clipped to the image (an empty block gives no entries)
    const int bx0 = txi * kTile + ((warp & 1) << 3), by0 = tyi * kTile + ((warp >> 1) << 2);
    uint32_t n_over = 0;
    FootPending P;
    s_img[0][tid] = 0.f;
    s_img[1][tid] = 0.f;
    s_img[2][tid] = 0.f;
    s_img[3][tid] = 1.f;
    const bool cull = pC == nullptr || vp.cull_occluded != 0;   // as in blend_fwd_tile
    for (int r = 0; r < vp.K; ++r) {
        const int k = vp.order[r];
        const uint2 rg = ranges[r];
        const bool live = inside && want && !(cull && s_img[3][tid] < vp.eps_T);
        if (cull && __syncthreads_count(live) == 0) {
            if (inside && pC) {
                pC[((size_t)k * 3 + 0) * HW + pix] = 0.f;
                pC[((size_t)k * 3 + 1) * HW + pix] = 0.f;
                pC[((size_t)k * 3 + 2) * HW + pix] = 0.f;
                pT[(size_t)k * HW + pix] = 1.f;
            }
            continue;
        }
        if (threadIdx.x == 0) leaf_path(tp, k, lp);   // read only after the next barrier
        float C0 = 0.f, C1 = 0.f, C2 = 0.f;
        float T = live ? 1.f : 0.f;
        bool frozen = !live;
        int ph = 0, pn = 0;
        float hs = kInfF;
        const float Pf = s_img[3][tid];   // transmittance in front of the subset
        const float gC0 = gI0 * Pf, gC1 = gI1 * Pf, gC2 = gI2 * Pf;
        // blends the nearest pending contributor (and, backward, adds its adjoint first)
        auto pop = [&]() {
            if (kBwd) {
                const uint32_t id = P.id[ph];
                pair_adjoint_add(rec, id, P.sig[ph], T, rec[3 * (size_t)id + 2], gC0, gC1, gC2, qf, acc, pcx, pcy,
                                 x0, y0, vp.alpha_max, g2d);
            }
            foot_pop(P, rec, ph, pn, hs, C0, C1, C2, T);
        };
        for (uint32_t b0 = rg.x; b0 < rg.y; b0 += kBlendThreads) {
            const int nb = (int)min((uint32_t)kBlendThreads, rg.y - b0);
            __syncthreads();
            if ((int)threadIdx.x < nb) {
                const uint32_t id = ival[b0 + threadIdx.x];
                StagedRec sr = stage_record(rec, id, x0, y0, vp);
                const float4 r0 = rec[3 * (size_t)id];
                const float4 sd = side[id];
                smask[threadIdx.x] =
                    sr.b.z >= 0.f ? foot_block_mask(sr, vp, k, foot_depth_radius(sr.c.w, sd.x), x0, y0) : 0u;
                srec[threadIdx.x] = sr;
                sbound[threadIdx.x] = foot_bound(r0.x, r0.y, sr.c.w, txi, tyi, vp);
                sctr[threadIdx.x] = make_float4(r0.x, r0.y, sr.c.w, 0.f);
                float bh, bl, dh, dl;
                two_sum(r0.x, -vp.cx, bh, bl);
                two_sum(r0.y, -vp.cy, dh, dl);
                skey[threadIdx.x] = make_float4(bh, __fadd_rn(bl, sd.z), dh, __fadd_rn(dl, sd.w));
                sextra[threadIdx.x] = make_float2(sd.x, sd.y);
                sid[threadIdx.x] = id;
            }
            __syncthreads();
            const int n = warp_list<false>(smask, nb, warp, lane, wl);
            {
                // block bounds of the warp's entries, then their suffix minimum, back to front
                const float cap = sbound[nb - 1];
                float carry = cap;
                for (int c = ((n - 1) >> 5) << 5; c >= 0; c -= 32) {
                    const int t = c + lane;
                    float v = kInfF;
                    if (t < n) {
                        const float4 m = sctr[wl[t]];
                        v = fmaxf(foot_bound_px(m.x, m.y, m.z, bx0, bx0 + 7, by0, by0 + 3, vp), sbound[wl[t]]);
                    }
                    // suffix minimum within the chunk (lanes above hold later entries)
                    for (int o = 1; o < 32; o <<= 1) {
                        const float w = __shfl_down_sync(0xffffffffu, v, o);
                        if (lane + o < 32) v = fminf(v, w);
                    }
                    v = fminf(v, carry);
                    if (t < n) wthr[warp][t] = v;
                    carry = __shfl_sync(0xffffffffu, v, 0);
                }
                __syncwarp();
            }
            for (int t0 = 0; t0 < n; t0 += 32) {
                if (!frozen && T < vp.eps_T) {
                    frozen = true;
                    s_tkeep[tid] = T;
                    T = 0.f;
                    pn = 0;
                    hs = kInfF;
                }
                if (__all_sync(0xffffffffu, frozen)) break;
                const int t1 = min(n, t0 + 32);
                for (int t = t0; t < t1; ++t) {
                    const int j = wl[t];
                    const float bound = wthr[warp][t];
                    // nothing from here on can come before a pending key below this bound
                    while (hs < bound) pop();
                    const float4 A = srec[j].a;
                    const float4 B = srec[j].b;
                    const float4 Cc = srec[j].c;
                    const float4 Kb = skey[j];
                    const float2 ex = sextra[j];
                    const float dx = pcx - A.x, dy = pcy - A.y;
                    const float u1 = fmaf(A.z, dx, A.w * dy), u2 = B.x * dy;
                    const float d2 = fmaf(u1, u1, u2 * u2);
                    const float ux = Kb.x * vp.ifx, uy = Kb.z * vp.ify;
                    const float bx = dx * vp.ifx, by = dy * vp.ify;
                    const float cr = fmaf(ux, by, -uy * bx);
                    // the ball test at the foot: |x_i - u_i|^2 / z^2 = (bx^2 + by^2 + cr^2) / |r_p|^2
                    bool ok = (d2 <= B.z) & (fmaf(bx, bx, fmaf(by, by, cr * cr)) <= ex.x * r2);
                    if (B.w < 0.f) {   // warp-uniform: Eq. 6 at the foot, with the key in one float
                        const float s1 = Cc.w * fmaf(pa, Kb.x, fmaf(pc, Kb.z, sc.x));
                        ok = ok && in_subset_foot(lp, vp.L, s1 * izf, g0, g1, g2, vp);
                    }
                    if (ok && !frozen) {
                        // s = z (fx^2 + a b + k c d) as a float pair
                        float p1, e1, p2, e2, q1, t1, q2, t2, Sh, Sl, kh, kl;
                        two_prod(pa, Kb.x, p1, e1);
                        e1 = __fmaf_rn(pa, Kb.y, e1);
                        two_prod(pc, Kb.z, p2, e2);
                        e2 = __fmaf_rn(pc, Kb.w, e2);
                        two_sum(Fh, p1, q1, t1);
                        two_sum(q1, p2, q2, t2);
                        fast_two_sum(q2, __fadd_rn(__fadd_rn(__fadd_rn(t1, t2), __fadd_rn(e1, e2)), Fl), Sh, Sl);
                        two_prod(Cc.w, Sh, kh, kl);
                        kl = __fmaf_rn(Cc.w, Sl, __fmaf_rn(ex.y, Sh, kl));
                        fast_two_sum(kh, kl, kh, kl);
                        const float G = ex2_approx(d2 * kNegHalfLog2e);
                        const float sig = fminf(B.y * G, vp.alpha_max);
                        if (pn == kFootPend) {   // full: the nearest is blended early
                            pop();
                            ++n_over;
                        }
                        foot_insert(P, rec, ph, pn, hs, kh, kl, sig, sid[j], C0, C1, C2, T, n_over);
                    }
                }
            }
            if (__syncthreads_count(frozen || T < vp.eps_T) == kBlendThreads) break;
        }
        while (pn > 0) pop();
        if (frozen && inside) T = live ? s_tkeep[tid] : 1.f;
        if (inside) {
            if (pC) {
                pC[((size_t)k * 3 + 0) * HW + pix] = C0;
                pC[((size_t)k * 3 + 1) * HW + pix] = C1;
                pC[((size_t)k * 3 + 2) * HW + pix] = C2;
                pT[(size_t)k * HW + pix] = T;
            }
            const float Pm = s_img[3][tid];
            s_img[0][tid] = fmaf(C0, Pm, s_img[0][tid]);
            s_img[1][tid] = fmaf(C1, Pm, s_img[1][tid]);
            s_img[2][tid] = fmaf(C2, Pm, s_img[2][tid]);
            s_img[3][tid] = Pm * T;
        }
    }
    if (!kBwd && inside && image) {
        const float Pm = s_img[3][tid];
        image[0 * HW + pix] = fmaf(vp.bg[0], Pm, s_img[0][tid]);
        image[1 * HW + pix] = fmaf(vp.bg[1], Pm, s_img[1][tid]);
        image[2 * HW + pix] = fmaf(vp.bg[2], Pm, s_img[2][tid]);
        if (Tfin) Tfin[pix] = Pm;
    }
    count_add(over, n_over);
}

// ------------------------------------------------------------------ blend backward

// kFlat = false: the adjoint of Eq. 5 and each subset's replay from its stored partials
// (pC, pT; `img` unused).  kFlat = true: the adjoint of the flat form (Eq. 2, which Eq. 5
// equals exactly: appendix proof) from the merged image alone (`img`; pC, pT unused): one
// front-to-back replay of the tile's concatenated subset-ordered list per pixel, with the
// transmittance in front of each subset (P) rebuilt from the replayed subset ends, and
// dL/dsigma_i = T_i <g, c_i> - <g, C - A_i> / (1 - sigma_i) where C is the image and A_i the
// colour blended up to and including pair i (both global).
//
// One tile of the view (the whole block calls it): `ranges` points at the tile's K runs
// (view rank order); payloads are record indices into rec and g2d (>= n_splats: skipped).
template <bool kCount, bool kFlat>
__device__ __forceinline__ void blend_bwd_tile(const ViewParams& vp, const TreeParams& tp, int tile,
                                               const uint2* __restrict__ ranges, const uint32_t* __restrict__ ival,
                                               const float4* __restrict__ rec, const float* __restrict__ pC,
                                               const float* __restrict__ pT, const float* __restrict__ img,
                                               const float* __restrict__ gI, float4* __restrict__ g2d,
                                               uint32_t n_inst, uint32_t n_splats,
                                               unsigned long long* __restrict__ pairs) {
    // <g, S_r> of this pixel for every rank: private to the thread, in local memory (cached),
    // so that shared memory does not grow with K (the flat form needs none)
    float behind_r[kFlat ? 1 : 1 << kMaxRenderDepth];
    uint32_t n_eval = 0, n_contrib = 0, n_iter = 0;
    __shared__ StagedRec srec[kBlendThreads];
    __shared__ uint32_t smask[kBlendThreads];
    __shared__ float4 splane[kBlendThreads][kMaxCutPlanes];
    __shared__ float sacc[kBlendThreads][9];
    __shared__ uint8_t wlist[kBlendThreads / 32][kBlendThreads];
    __shared__ LeafPath lp;
    // per warp, the (pixel, entry) scalars of the current stretch of kBwdSub list entries
    __shared__ float sh_h[kBlendThreads / 32][32 * kBwdSubPad];   // sigma dL/dsigma
    __shared__ float sh_w[kBlendThreads / 32][32 * kBwdSubPad];   // sigma T
    __shared__ float4 s_gc[kBlendThreads];                          // dL/dC_k of each pixel (w unused)
    const int tyi = tile / vp.tiles_x, txi = tile - tyi * vp.tiles_x;
    int lx, ly;
    thread_pixel(threadIdx.x, lx, ly);
    const int warp = threadIdx.x >> 5;
    const int px = txi * kTile + lx, py = tyi * kTile + ly;
    const bool inside = px < vp.W && py < vp.H;
    const float x0 = (float)(txi * kTile), y0 = (float)(tyi * kTile);
    const float pcx = lx + 0.5f, pcy = ly + 0.5f;
    const int lane = threadIdx.x & 31;
    const float Xc = (float)px + 0.5f, Yc = (float)py + 0.5f;   // absolute pixel centre (Eq. 6 tests)
    const size_t HW = (size_t)vp.W * vp.H;
    const size_t pix = inside ? (size_t)py * vp.W + px : 0;
    uint8_t* wl = wlist[warp];
    const int wx0 = (warp & 1) << 3, wy0 = (warp >> 1) << 2;   // the warp's 8x4 block in the tile

    __syncthreads();   // a previous tile's readers of the shared arrays are done
    for (int i = threadIdx.x; i < kBlendThreads * 9; i += kBlendThreads) (&sacc[0][0])[i] = 0.f;

    // adjoint of Eq. 5: <g, S_r> for every rank, back to front
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (inside) {
        g0 = gI[0 * HW + pix];
        g1 = gI[1 * HW + pix];
        g2 = gI[2 * HW + pix];
    }
    if (!kFlat) {
        float behind = g0 * vp.bg[0] + g1 * vp.bg[1] + g2 * vp.bg[2];
        for (int r = vp.K - 1; r >= 0; --r) {
            behind_r[r] = behind;
            if (inside) {
                const int k = vp.order[r];
                float c0 = pC[((size_t)k * 3 + 0) * HW + pix], c1 = pC[((size_t)k * 3 + 1) * HW + pix],
                      c2 = pC[((size_t)k * 3 + 2) * HW + pix], t = pT[(size_t)k * HW + pix];
                behind = fmaf(t, behind, g0 * c0 + g1 * c1 + g2 * c2);
            }
        }
    }
    // flat form: <g, C> of the whole pixel, and the colour blended so far (acc) carried over
    // subsets
    const float qflat = kFlat && inside ? g0 * img[0 * HW + pix] + g1 * img[1 * HW + pix] + g2 * img[2 * HW + pix]
                                        : 0.f;
    float acc = 0.f;   // <gC, colour blended so far> (per subset; over all subsets in the flat form)
    float Pm = 1.f;
    for (int r = 0; r < vp.K; ++r) {
        const int k = vp.order[r];
        float Ck0 = 0.f, Ck1 = 0.f, Ck2 = 0.f, Tk = 1.f;
        if (!kFlat && inside) {
            Ck0 = pC[((size_t)k * 3 + 0) * HW + pix];
            Ck1 = pC[((size_t)k * 3 + 1) * HW + pix];
            Ck2 = pC[((size_t)k * 3 + 2) * HW + pix];
            Tk = pT[(size_t)k * HW + pix];
        }
        const float gC0 = g0 * Pm, gC1 = g1 * Pm, gC2 = g2 * Pm;
        s_gc[threadIdx.x] = make_float4(gC0, gC1, gC2, 0.f);   // read by this warp's lanes after the next barrier
        // q - acc = <g, colour behind the current pair> (times P for the per-subset form)
        float q;
        if (kFlat) {
            q = qflat;
        } else {
            const float gT = Pm * behind_r[r];
            q = gC0 * Ck0 + gC1 * Ck1 + gC2 * Ck2 + gT * Tk;
            acc = 0.f;
        }
        // a pixel whose transmittance in front of this subset is below eps_T gets gradients
        // scaled by less than eps_T from it: the subset is skipped there, as an image-only
        // forward skips it
        const bool front_open = Pm >= vp.eps_T;
        if (!kFlat) Pm *= Tk;
        if (threadIdx.x == 0) leaf_path(tp, k, lp);   // read only after the next barrier
        uint2 rg = ranges[r];
        rg.y = min(rg.y, n_inst);   // lists handed over from a forward: never read past them
        rg.x = min(rg.x, rg.y);
        const bool active = inside && front_open && (g0 != 0.f || g1 != 0.f || g2 != 0.f);
        // an inactive pixel stays inactive for every later subset (P only falls): nothing of
        // the tile is left to replay once all are
        if (__syncthreads_count(active) == 0) break;
        // replay of the forward: the same pairs, the same freeze points (an inactive pixel
        // is frozen from the start, with q = acc: its pairs get zero gradients)
        bool frozen = !active;
        float T = active ? 1.f : 0.f;
        float Tkeep = 1.f;     // transmittance of the subset where the pixel froze (flat form)
        const float qkeep = q;
        if (!active) q = acc;
        for (uint32_t b0 = rg.x; b0 < rg.y; b0 += kBlendThreads) {
            const int nb = (int)min((uint32_t)kBlendThreads, rg.y - b0);
            __syncthreads();
            if ((int)threadIdx.x < nb) {
                StagedRec sr;
                uint32_t msk;
                uint32_t id = ival[b0 + threadIdx.x];
                if (id < n_splats) {
                    stage_for_subset(rec, id, x0, y0, vp, lp, sr, msk, splane[threadIdx.x]);
                } else {   // not a splat: touches no pixel
                    id = 0;
                    msk = 0u;
                    sr.a = sr.b = sr.c = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                srec[threadIdx.x] = sr;
                smask[threadIdx.x] = msk;
            }
            __syncthreads();
            const int n = warp_list<false>(smask, nb, warp, lane, wl);
            for (int t0 = 0; t0 < n; t0 += 32) {
                if (!frozen && T < vp.eps_T) {
                    // frozen as in the forward: later pairs get sigma * T = 0, and q = acc
                    // makes their adjoint vanish too
                    frozen = true;
                    Tkeep = T;
                    T = 0.f;
                    q = acc;
                }
                if (__all_sync(0xffffffffu, frozen)) break;
                const int t1 = min(n, t0 + 32);
                for (int s0 = t0; s0 < t1; s0 += kBwdSub) {
                    const int s1 = min(t1, s0 + kBwdSub);
                    // phase 1, pixel by pixel: the forward's arithmetic, then the adjoint of
                    // the pair with the same predicate (a pair that fails gets sigma = 0 and
                    // zero gradients); two scalars per (pixel, entry) go to shared memory
                    auto pair = [&](int t, int e) {
                        if (kCount && lane == 0) ++n_iter;
                        const int j = wl[t];
                        const float4 A = srec[j].a;
                        const float4 B = srec[j].b;
                        const float4 Cc = srec[j].c;
                        const float dx = pcx - A.x, dy = pcy - A.y;
                        const float u1 = fmaf(A.z, dx, A.w * dy), u2 = B.x * dy;
                        const float d2 = fmaf(u1, u1, u2 * u2);
                        const float G = ex2_approx(d2 * kNegHalfLog2e);
                        const float raw = B.y * G;
                        bool ok;
                        float sig;
                        const float w_T = T;
                        const float grgb = gC0 * Cc.x + gC1 * Cc.y + gC2 * Cc.z;
                        float h;
                        if (B.w == kInfF) {   // warp-uniform: the Mahalanobis test alone, no clamp
                            ok = d2 <= B.z;
                            sig = ok ? raw : 0.f;
                            const float w = sig * w_T;
                            acc = fmaf(w, grgb, acc);
                            // a failing pair has sigma = 0, so h = 0 with no select
                            h = sig * (w_T * grgb - __fdividef(q - acc, 1.f - sig));
                            sh_w[warp][lane * kBwdSubPad + e] = w;
                        } else {
                            ok = pair_passes(B, Cc, dx, dy, d2, splane[j], smask[j], vp, lp, Xc, Yc);
                            const bool grad = ok && raw < vp.alpha_max;
                            sig = ok ? fminf(raw, vp.alpha_max) : 0.f;
                            const float w = sig * w_T;
                            acc = fmaf(w, grgb, acc);
                            const float dsig = w_T * grgb - __fdividef(q - acc, 1.f - sig);
                            h = grad ? sig * dsig : 0.f;   // sigma dL/dsigma
                            sh_w[warp][lane * kBwdSubPad + e] = w;
                        }
                        if (kCount && !frozen) {
                            ++n_eval;
                            n_contrib += ok;
                        }
                        sh_h[warp][lane * kBwdSubPad + e] = h;
                        T = fmaf(-sig, T, T);
                    };
                    if (s1 - s0 == kBwdSub) {   // a full stretch: fixed shared-memory offsets
#pragma unroll 2
                        for (int e = 0; e < kBwdSub; ++e) pair(s0 + e, e);
                    } else {
                        for (int t = s0; t < s1; ++t) pair(t, t - s0);
                    }
                    __syncwarp();
                    // phase 2, record by record: lane (half g of the warp's block, entry e)
                    // sums rows 2g and 2g + 1 (8 pixels each).  With delta = (dx, dy) from the
                    // centre, u = L delta, h = sigma dL/dsigma, the pair's 2D gradients are
                    //   mean: h L^T u,  conic: -h/2 (dx^2, 2 dx dy, dy^2),  alpha: h / alpha,
                    //   colour: dL/dC_k sigma T,
                    // and dy is the same on a row, so three running sums in dx per row do.
                    const int g = lane >> 4, e = lane & 15;
                    float o[9];
#pragma unroll
                    for (int c = 0; c < 9; ++c) o[c] = 0.f;
                    int jr = 0;
                    if (s0 + e < s1) {
                        jr = wl[s0 + e];
                        const float4 A = srec[jr].a;
                        const float4 B = srec[jr].b;
                        const float dx0 = ((float)wx0 + 0.5f) - A.x;
                        float Sh_all = 0.f;
#pragma unroll
                        for (int row = 2 * g; row < 2 * g + 2; ++row) {
                            const float dy = ((float)(wy0 + row) + 0.5f) - A.y;
                            float Sh = 0.f, Shx = 0.f, Shxx = 0.f;
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const int p = row * 8 + i;
                                const float h = sh_h[warp][p * kBwdSubPad + e], w = sh_w[warp][p * kBwdSubPad + e];
                                const float dx = dx0 + (float)i;
                                const float hdx = h * dx;
                                Sh += h;
                                Shx += hdx;
                                Shxx = fmaf(hdx, dx, Shxx);
                                const float4 gc = s_gc[warp * 32 + p];
                                o[6] = fmaf(gc.x, w, o[6]);
                                o[7] = fmaf(gc.y, w, o[7]);
                                o[8] = fmaf(gc.z, w, o[8]);
                            }
                            const float shu1 = fmaf(A.z, Shx, A.w * dy * Sh);   // row sum of h u1
                            o[0] = fmaf(A.z, shu1, o[0]);
                            o[1] += fmaf(A.w, shu1, B.x * B.x * dy * Sh);
                            o[2] = fmaf(-0.5f, Shxx, o[2]);
                            o[3] = fmaf(-dy, Shx, o[3]);
                            o[4] = fmaf(-0.5f * dy * dy, Sh, o[4]);
                            Sh_all += Sh;
                        }
                        o[5] = __fdividef(Sh_all, B.y);
                    }
                    // the two halves of an entry: lanes e and e + 16
#pragma unroll
                    for (int c = 0; c < 9; ++c) o[c] += __shfl_xor_sync(0xffffffffu, o[c], 16);
                    if (g == 0 && s0 + e < s1) {
#pragma unroll
                        for (int c = 0; c < 9; ++c) atomicAdd(&sacc[jr][c], o[c]);
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            if ((int)threadIdx.x < nb) {
                float* a = sacc[threadIdx.x];
                bool nz = false;
                for (int t = 0; t < 9; ++t) nz |= a[t] != 0.f;
                const uint32_t id = ival[b0 + threadIdx.x];
                if (nz && id < n_splats) {
                    float4* dst = g2d + 3 * (size_t)id;
                    red_add_v4(dst, make_float4(a[0], a[1], a[2], a[3]));
                    red_add_v4(dst + 1, make_float4(a[4], a[5], a[6], a[7]));
                    red_add_v4(dst + 2, make_float4(a[8], 0.f, 0.f, 0.f));
                    for (int t = 0; t < 9; ++t) a[t] = 0.f;
                }
            }
            if (__syncthreads_count(frozen || T < vp.eps_T) == kBlendThreads) break;
        }
        if (kFlat && active) {
            // the subset's end transmittance, as the forward stored it: P in front of the next
            Pm *= frozen ? Tkeep : T;
            q = qkeep;   // undo a freeze's q = acc: later subsets see the whole pixel again
        }
    }
    if (kCount) {
        count_pairs(pairs + 2, n_eval, n_contrib);
        count_add(pairs + 12, n_iter);
    }
}

template <bool kCount, bool kFlat>
__global__ void __launch_bounds__(kBlendThreads, RGS_BLEND_MIN_BLOCKS)
blend_bwd_kernel(ViewParams vp, TreeParams tp, const uint2* __restrict__ ranges, const uint32_t* __restrict__ ival,
                 const float4* __restrict__ rec, const float* __restrict__ pC, const float* __restrict__ pT,
                 const float* __restrict__ img, const float* __restrict__ gI, float4* __restrict__ g2d,
                 uint32_t n_inst, uint32_t n_splats, unsigned long long* __restrict__ pairs) {
    blend_bwd_tile<kCount, kFlat>(vp, tp, blockIdx.x, ranges + (size_t)blockIdx.x * vp.K, ival, rec, pC, pT, img,
                                  gI, g2d, n_inst, n_splats, pairs);
}

// Flat backward of a batch of views (a training step over several views), persistent over
// the batch's global tiles like blend_batch_kernel: each block takes the next tile from a
// device counter (counters[7]); the slot's image and dL/dimage come from its BatchSlot and
// the payloads index the batch's per-(slot, splat) records and 2D-gradient records.
template <bool kCount>
__global__ void __launch_bounds__(kBlendThreads, RGS_BLEND_MIN_BLOCKS)
blend_bwd_batch_kernel(const BatchSlot* __restrict__ slots, const BatchHeader* __restrict__ hdr, TreeParams tp,
                       const uint2* __restrict__ ranges, const uint32_t* __restrict__ ival,
                       const float4* __restrict__ rec, float4* __restrict__ g2d, uint32_t n_inst, uint32_t n_splats,
                       unsigned long long* __restrict__ counters, unsigned long long* __restrict__ pairs) {
    __shared__ ViewParams svp;
    __shared__ uint32_t s_tile;
    __shared__ int s_slot;
    const int S = hdr->S;
    const uint32_t total = hdr->total_tiles;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t t = (uint32_t)atomicAdd(&counters[7], 1ull);
            int sl = 0;
            while (sl + 1 < S && hdr->tile_base[sl + 1] <= t) ++sl;
            s_tile = t;
            s_slot = sl;
        }
        __syncthreads();
        const uint32_t t = s_tile;
        const int slot = s_slot;
        if (t >= total) break;
        if (slot != cur) {
            constexpr int kWords = (int)(sizeof(ViewParams) / 4);
            for (int w = threadIdx.x; w < kWords; w += blockDim.x)
                reinterpret_cast<uint32_t*>(&svp)[w] = reinterpret_cast<const uint32_t*>(&slots[slot].vp)[w];
            cur = slot;
            __syncthreads();
        }
        blend_bwd_tile<kCount, true>(svp, tp, (int)(t - hdr->tile_base[slot]), ranges + (size_t)t * svp.K, ival, rec,
                                     nullptr, nullptr, slots[slot].image, slots[slot].grad, g2d, n_inst, n_splats,
                                     pairs);
        __syncthreads();   // s_tile is rewritten by the next claim
    }
}

// ------------------------------------------------------------------ standalone merge (Eq. 5)
__global__ void merge_kernel(const float* __restrict__ pC, const float* __restrict__ pT,
                             const int32_t* __restrict__ order, int K, int64_t HW, float bg0, float bg1, float bg2,
                             float* __restrict__ image, float* __restrict__ Tout) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= HW) return;
    float c0 = 0.f, c1 = 0.f, c2 = 0.f, P = 1.f;
    for (int r = 0; r < K; ++r) {
        const int64_t k = order[r];
        c0 = fmaf(pC[(k * 3 + 0) * HW + i], P, c0);
        c1 = fmaf(pC[(k * 3 + 1) * HW + i], P, c1);
        c2 = fmaf(pC[(k * 3 + 2) * HW + i], P, c2);
        P *= pT[k * HW + i];
    }
    image[0 * HW + i] = fmaf(bg0, P, c0);
    image[1 * HW + i] = fmaf(bg1, P, c1);
    image[2 * HW + i] = fmaf(bg2, P, c2);
    if (Tout) Tout[i] = P;
}

// Adjoint of Eq. 5 per pixel: a back-to-front pass gives <g, S_r> and the suffix products,
// a front-to-back pass the prefix products.
__global__ void merge_bwd_kernel(const float* __restrict__ pC, const float* __restrict__ pT,
                                 const int32_t* __restrict__ order, int K, int64_t HW, float bg0, float bg1,
                                 float bg2, const float* __restrict__ gI, const float* __restrict__ gTo,
                                 float* __restrict__ dC, float* __restrict__ dT) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= HW) return;
    const float g0 = gI[i], g1 = gI[HW + i], g2 = gI[2 * HW + i];
    const float gt = gTo ? gTo[i] : 0.f;
    // back to front: dT_k <- <g, S_r> and the suffix product behind r (stored temporarily)
    float behind = g0 * bg0 + g1 * bg1 + g2 * bg2, suffix = 1.f;
    for (int r = K - 1; r >= 0; --r) {
        const int64_t k = order[r];
        dT[k * HW + i] = behind;
        dC[(k * 3) * HW + i] = suffix;
        const float t = pT[k * HW + i];
        behind = fmaf(t, behind, g0 * pC[(k * 3) * HW + i] + g1 * pC[(k * 3 + 1) * HW + i] + g2 * pC[(k * 3 + 2) * HW + i]);
        suffix *= t;
    }
    float P = 1.f;
    for (int r = 0; r < K; ++r) {
        const int64_t k = order[r];
        const float suf = dC[(k * 3) * HW + i];
        dT[k * HW + i] = P * dT[k * HW + i] + gt * P * suf;
        dC[(k * 3 + 0) * HW + i] = g0 * P;
        dC[(k * 3 + 1) * HW + i] = g1 * P;
        dC[(k * 3 + 2) * HW + i] = g2 * P;
        P *= pT[k * HW + i];
    }
}

}  // namespace

int launch_emit(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* sorted_ids,
                int64_t n_vis, cudaStream_t s) {
    if (n_vis <= 0) return RGS_OK;
    const int64_t want = (n_vis + 255) / 256;      // one warp per 32 splats
    const int64_t cap = (int64_t)sm_count() * 16;                  // grid-stride beyond: amortises the tree copy
    unsigned grid = (unsigned)(want < cap ? want : cap);
    // work counters (zeroed with the others at the start of the list build): [4], [5] the
    // emission queues, [8], [9] the splats each launch deferred, [12] the items the count kept
    auto queues_of = [&](int multi) {
        EmitQueues q;
        q.list = b.units ? reinterpret_cast<uint2*>(b.units) + (size_t)multi * b.unit_cap : nullptr;
        q.count = b.counters + 8 + multi;
        q.cap = b.units ? b.unit_cap : 0u;
        return q;
    };
    const unsigned lgrid = (unsigned)sm_count() * 8;
    const uint32_t* item_at = b.items ? b.item_at : nullptr;
    const EmitQueues q0 = queues_of(0), q1 = queues_of(1);
    // foot reading: straddlers are clipped over the foot's depth interval (side array)
    const float4* side = vp.foot ? b.foot_side : nullptr;
    // 1. splats of few items, the first instance of each splat whose items the count kept,
    //    and the list of the others
    emit_kernel<0><<<grid, 256, 0, s>>>(vp, tp, sorted_ids, n_vis, b.ioff, b.rect, b.mask, b.rec, b.cull, b.cull_chunk,
                                        b.ikey, b.ival, b.counters + 4, nullptr, q0, item_at, b.ibase);
    RGS_CUDA_LAUNCH_CHECK();
    if (vp.K > 1) {
        emit_kernel<1><<<grid, 256, 0, s>>>(vp, tp, sorted_ids, n_vis, b.ioff, b.rect, b.mask, b.rec, b.cull,
                                            b.cull_chunk, b.ikey, b.ival, b.counters + 5, side, q1, item_at, b.ibase);
        RGS_CUDA_LAUNCH_CHECK();
    }
    // 2. the kept items
    if (item_at) {
        emit_items_kernel<<<(unsigned)sm_count() * 8, 256, 0, s>>>(vp, b.items, b.item_first, b.item_ctr, b.item_cap, b.ibase,
                                                  b.rec, b.cull, b.cull_chunk, b.ikey, b.ival);
        RGS_CUDA_LAUNCH_CHECK();
    }
    // 3. the listed splats
    if (q0.list) {
        emit_listed_kernel<0><<<lgrid, 256, 0, s>>>(vp, tp, q0, b.rect, b.mask, b.rec, b.cull, b.cull_chunk, b.ikey,
                                                    b.ival, nullptr);
        RGS_CUDA_LAUNCH_CHECK();
        if (vp.K > 1) {
            emit_listed_kernel<1><<<lgrid, 256, 0, s>>>(vp, tp, q1, b.rect, b.mask, b.rec, b.cull, b.cull_chunk,
                                                        b.ikey, b.ival, side);
            RGS_CUDA_LAUNCH_CHECK();
        }
    }
    return RGS_OK;
}

int launch_cull_chunks(const ViewParams& vp, const float* cull, float2* chunk, cudaStream_t s) {
    const int64_t total = (int64_t)vp.tiles_y * ((vp.tiles_x + kCullChunk - 1) / kCullChunk) * vp.K;
    cull_chunk_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(vp, cull, chunk);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_ranges(const uint32_t* keys, int64_t n, uint2* ranges, int64_t n_ranges, cudaStream_t s, uint32_t first,
                  bool clear) {
    if (clear) RGS_CUDA_TRY(cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_ranges, s));
    if (n <= 0) return RGS_OK;
    const int64_t want = (n + 1023) / 1024, cap = (int64_t)sm_count() * 8;
    ranges_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(keys, n, ((uintptr_t)keys & 15) == 0,
                                                                            ranges, first);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_open_prefix(const ViewParams& vp, const uint8_t* open, uint32_t* prefix, uint32_t* sat, cudaStream_t s) {
    const unsigned grid = (unsigned)((vp.tiles_y + 7) / 8);
    open_prefix_kernel<<<grid, 256, 0, s>>>(open, vp.tiles_x, vp.tiles_y, prefix);
    RGS_CUDA_LAUNCH_CHECK();
    open_sat_kernel<<<(unsigned)((vp.tiles_x + 1 + 255) / 256), 256, 0, s>>>(prefix, vp.tiles_x, vp.tiles_y, sat);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_recount(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* sorted_ids,
                   int64_t n_vis, uint32_t* cnt_out, cudaStream_t s) {
    if (n_vis <= 0) return RGS_OK;
    const int64_t want = (n_vis + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 16;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    recount_kernel<false><<<grid, 256, 0, s>>>(vp, nullptr, nullptr, 0, tp, sorted_ids, n_vis, nullptr, nullptr,
                                               b.rect, b.mask, b.rec, b.item_at, b.items, b.items ? b.item_cap : 0u,
                                               cnt_out, b.counters + 4, b.counters + 15);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_blend_fwd(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* ival,
                     float* partial_C, float* partial_T, float* image, float* T_final, float* tile_depth,
                     cudaStream_t s, bool record_ends, int r_begin, int r_end) {
    if (r_end < 0) r_end = vp.K;
    if ((r_begin > 0 || r_end < vp.K) && (partial_C || !b.state || !b.open)) {
        set_error("blend: ranks blended in groups need an image-only render and the group state buffers");
        return RGS_EINVAL;
    }
    unsigned grid = (unsigned)(vp.tiles_x * vp.tiles_y);
    unsigned long long* pairs = prof_pair_counters();
    if (pairs)
        blend_fwd_kernel<true><<<grid, kBlendThreads, 0, s>>>(vp, tp, b.ranges, ival, b.rec, partial_C, partial_T, image,
                                                              T_final, tile_depth, record_ends, pairs, r_begin, r_end,
                                                              b.state, b.open, nullptr);
    else
        blend_fwd_kernel<false><<<grid, kBlendThreads, 0, s>>>(vp, tp, b.ranges, ival, b.rec, partial_C, partial_T,
                                                               image, T_final, tile_depth, record_ends, nullptr,
                                                               r_begin, r_end, b.state, b.open, nullptr);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

// One request of a batch blended as its own launch of blend_fwd_kernel (its view a kernel
// parameter): the argument list of that launch, and its launch during a stream capture or
// the update of its graph node for the next batch.
namespace {
struct BlendNodeParams {
    void* args[17];
    bool record_ends = false;
    unsigned long long* pairs = nullptr;
    float *pC = nullptr, *pT = nullptr, *Tfin = nullptr, *tile_depth = nullptr;
    BlendNodeArgs a;
    explicit BlendNodeParams(const BlendNodeArgs& x) : a(x) {
        void* p[17] = {&a.vp,    &a.tp,         &a.ranges,      &a.ival,  &a.rec,     &pC,     &pT,      &a.image, &Tfin,
                       &tile_depth, &record_ends, &pairs, &a.r_begin, &a.r_end, &a.state, &a.open, &a.skip};
        for (int i = 0; i < 17; ++i) args[i] = p[i];
    }
    cudaKernelNodeParams node(unsigned grid) {
        cudaKernelNodeParams k;
        memset(&k, 0, sizeof k);
        k.func = (void*)blend_fwd_kernel<false>;
        k.gridDim = dim3(grid > 0 ? grid : 1u);
        k.blockDim = dim3(kBlendThreads);
        k.sharedMemBytes = 0;
        k.kernelParams = args;
        return k;
    }
};
}  // namespace

int launch_blend_node(const BlendNodeArgs& a, unsigned grid, cudaStream_t s) {
    blend_fwd_kernel<false><<<grid > 0 ? grid : 1u, kBlendThreads, 0, s>>>(
        a.vp, a.tp, a.ranges, a.ival, a.rec, nullptr, nullptr, a.image, nullptr, nullptr, false, nullptr, a.r_begin,
        a.r_end, a.state, a.open, a.skip);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int set_blend_node(cudaGraphExec_t exec, cudaGraphNode_t node, const BlendNodeArgs& a, unsigned grid) {
    BlendNodeParams p(a);
    const cudaKernelNodeParams k = p.node(grid);
    RGS_CUDA_TRY(cudaGraphExecKernelNodeSetParams(exec, node, &k));
    return RGS_OK;
}

int launch_foot_order(const ViewParams& vp, const RasterBuffers& b, int64_t I, cudaStream_t s,
                      const uint32_t** keys_out, const uint32_t** vals_out) {
    if (I <= 0) {
        *keys_out = b.ikey;
        *vals_out = b.ival;
        return RGS_OK;
    }
    const int64_t want = (I + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 16;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    foot_keys_kernel<<<grid, 256, 0, s>>>(vp, b.ikey, b.ival, I, b.rec, b.fkey, b.fidx);
    RGS_CUDA_LAUNCH_CHECK();
    // LSD: the bound first, then stably the (tile, subset) key
    bool alt = false;
    int rc = radix_sort_pairs(b.fkey, b.fidx, b.ikey_alt, b.ival_alt, I, 32, b.temp, b.temp_bytes, s, &alt);
    if (rc) return rc;
    const uint32_t* idx = alt ? b.ival_alt : b.fidx;
    uint32_t* k2 = alt ? b.fkey : b.ikey_alt;
    uint32_t* v2 = alt ? b.fidx : b.ival_alt;
    foot_gather_kernel<<<grid, 256, 0, s>>>(idx, I, b.ikey, b.ival, k2, v2);
    RGS_CUDA_LAUNCH_CHECK();
    bool alt2 = false;
    rc = radix_sort_pairs(k2, v2, b.ikey, b.ival, I, vp.tile_bits + vp.L, b.temp, b.temp_bytes, s, &alt2);
    if (rc) return rc;
    *keys_out = alt2 ? b.ikey : k2;
    *vals_out = alt2 ? b.ival : v2;
    return RGS_OK;
}

int launch_blend_foot(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* ival,
                      float* partial_C, float* partial_T, float* image, float* T_final,
                      unsigned long long* over, cudaStream_t s) {
    unsigned grid = (unsigned)(vp.tiles_x * vp.tiles_y);
    blend_foot_kernel<false><<<grid, kBlendThreads, 0, s>>>(vp, tp, b.ranges, ival, b.rec, b.foot_side, partial_C,
                                                            partial_T, image, T_final, over, nullptr, nullptr);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_blend_foot_bwd(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* ival,
                          const float* image, const float* dL_dimage, unsigned long long* over, cudaStream_t s) {
    unsigned grid = (unsigned)(vp.tiles_x * vp.tiles_y);
    blend_foot_kernel<true><<<grid, kBlendThreads, 0, s>>>(vp, tp, b.ranges, ival, b.rec, b.foot_side, nullptr,
                                                           nullptr, const_cast<float*>(image), nullptr, over,
                                                           dL_dimage, b.g2d);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_emit_batch(const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp, const RasterBuffers& b,
                      const uint32_t* sorted_ids, int64_t n_cap, int64_t N, unsigned long long* counters,
                      cudaStream_t s, const unsigned long long* inst_base, bool open_tables) {
    const uint32_t* item_at = b.items ? b.item_at : nullptr;
    emit_batch_kernel<0><<<(unsigned)sm_count() * 8, 256, 0, s>>>(slots, hdr, tp, sorted_ids, n_cap, N, counters, b.ioff, b.rect,
                                                 b.mask, b.rec, b.ikey, b.ival, item_at, b.ibase, inst_base);
    RGS_CUDA_LAUNCH_CHECK();
    if (tp.L > 0) {
        emit_batch_kernel<1><<<(unsigned)sm_count() * 8, 256, 0, s>>>(slots, hdr, tp, sorted_ids, n_cap, N, counters, b.ioff, b.rect,
                                                     b.mask, b.rec, b.ikey, b.ival, item_at, b.ibase, inst_base);
        RGS_CUDA_LAUNCH_CHECK();
    }
    if (item_at) {
        emit_items_batch_kernel<<<(unsigned)sm_count() * 8, 256, 0, s>>>(slots, hdr, b.items, b.item_ctr, b.item_cap, b.ibase, N,
                                                        counters, b.ikey, b.ival, inst_base, open_tables,
                                                        open_tables ? counters + kBatchBinCounter + 1 : nullptr);
        RGS_CUDA_LAUNCH_CHECK();
    }
    return RGS_OK;
}

int launch_ranges_dev(const uint32_t* keys, const unsigned long long* n_dev, int64_t cap, uint2* ranges,
                      cudaStream_t s, const unsigned long long* base_dev) {
    ranges_dev_kernel<<<(unsigned)sm_count() * 8, 256, 0, s>>>(keys, n_dev, cap, ranges, base_dev);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_blend_batch(const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp, uint2* ranges,
                       const uint32_t* ival, const float4* rec, unsigned long long* counters, cudaStream_t s,
                       bool record_ends) {
    int dev = 0, sms = 0;
    RGS_CUDA_TRY(cudaGetDevice(&dev));
    RGS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    blend_batch_kernel<<<(unsigned)(sms * RGS_BLEND_MIN_BLOCKS), kBlendThreads, 0, s>>>(slots, hdr, tp, ranges, ival,
                                                                                      rec, counters, record_ends);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_open_tables_batch(const BatchSlot* slots, const BatchHeader* hdr, const uint8_t* open, cudaStream_t s) {
    open_prefix_batch_kernel<<<dim3(16, kMaxSlots), 256, 0, s>>>(slots, hdr, open);
    RGS_CUDA_LAUNCH_CHECK();
    open_sat_batch_kernel<<<dim3(4, kMaxSlots), 256, 0, s>>>(slots, hdr);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_recount_batch(const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp, const RasterBuffers& b,
                         const uint32_t* sorted_ids, int64_t n_cap, int64_t N, unsigned long long* counters,
                         uint32_t* cnt_out, unsigned long long* queue, unsigned long long* total, cudaStream_t s) {
    ViewParams vp_unused;
    memset(&vp_unused, 0, sizeof vp_unused);
    recount_kernel<true><<<(unsigned)sm_count() * 8, 256, 0, s>>>(vp_unused, slots, hdr, N, tp, sorted_ids, n_cap, counters + 1,
                                                 counters + 2, b.rect, b.mask, b.rec, b.item_at, b.items,
                                                 b.items ? b.item_cap : 0u, cnt_out, queue, total);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_blend_bwd_batch(const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp, const uint2* ranges,
                           const uint32_t* ival, const float4* rec, float4* g2d, int64_t n_inst, int64_t n_splats,
                           unsigned long long* counters, cudaStream_t s) {
    int dev = 0, sms = 0;
    RGS_CUDA_TRY(cudaGetDevice(&dev));
    RGS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    static bool attr_set = false;
    if (!attr_set) {
        RGS_CUDA_TRY(cudaFuncSetAttribute(blend_bwd_batch_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared));
        RGS_CUDA_TRY(cudaFuncSetAttribute(blend_bwd_batch_kernel<false>,
                                          cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared));
        attr_set = true;
    }
    RGS_CUDA_TRY(cudaMemsetAsync(counters + 7, 0, 8, s));   // the work-queue head
    const unsigned grid = (unsigned)(sms * RGS_BLEND_MIN_BLOCKS);
    unsigned long long* pairs = prof_pair_counters();
    if (pairs)
        blend_bwd_batch_kernel<true><<<grid, kBlendThreads, 0, s>>>(slots, hdr, tp, ranges, ival, rec, g2d,
                                                                   (uint32_t)n_inst, (uint32_t)n_splats, counters,
                                                                   pairs);
    else
        blend_bwd_batch_kernel<false><<<grid, kBlendThreads, 0, s>>>(slots, hdr, tp, ranges, ival, rec, g2d,
                                                                    (uint32_t)n_inst, (uint32_t)n_splats, counters,
                                                                    nullptr);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_blend_bwd(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* ival,
                     const float* partial_C, const float* partial_T, const float* image, const float* dL_dimage,
                     int64_t n_inst, int64_t n_splats, cudaStream_t s) {
    unsigned grid = (unsigned)(vp.tiles_x * vp.tiles_y);
    const size_t smem = 0;
    static bool attr_set = false;
    if (!attr_set) {
        // about 58 KB per CTA: three CTAs per SM need most of the carveout as shared memory
        RGS_CUDA_TRY(cudaFuncSetAttribute(blend_bwd_kernel<true, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared));
        RGS_CUDA_TRY(cudaFuncSetAttribute(blend_bwd_kernel<false, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared));
        RGS_CUDA_TRY(cudaFuncSetAttribute(blend_bwd_kernel<true, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared));
        RGS_CUDA_TRY(cudaFuncSetAttribute(blend_bwd_kernel<false, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cudaSharedmemCarveoutMaxShared));
        attr_set = true;
    }
    unsigned long long* pairs = prof_pair_counters();
    const bool flat = image != nullptr;
    const uint32_t ni = (uint32_t)n_inst, ns = (uint32_t)n_splats;
    if (flat && pairs)
        blend_bwd_kernel<true, true><<<grid, kBlendThreads, smem, s>>>(vp, tp, b.ranges, ival, b.rec, nullptr, nullptr,
                                                                       image, dL_dimage, b.g2d, ni, ns, pairs);
    else if (flat)
        blend_bwd_kernel<false, true><<<grid, kBlendThreads, smem, s>>>(vp, tp, b.ranges, ival, b.rec, nullptr, nullptr,
                                                                        image, dL_dimage, b.g2d, ni, ns, nullptr);
    else if (pairs)
        blend_bwd_kernel<true, false><<<grid, kBlendThreads, smem, s>>>(vp, tp, b.ranges, ival, b.rec, partial_C,
                                                                        partial_T, nullptr, dL_dimage, b.g2d, ni, ns,
                                                                        pairs);
    else
        blend_bwd_kernel<false, false><<<grid, kBlendThreads, smem, s>>>(vp, tp, b.ranges, ival, b.rec, partial_C,
                                                                         partial_T, nullptr, dL_dimage, b.g2d, ni, ns,
                                                                         nullptr);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_merge(const float* pC, const float* pT, const int32_t* order, int K, int H, int W, const float bg[3],
                 float* image, float* T_out, cudaStream_t s) {
    int64_t HW = (int64_t)H * W;
    merge_kernel<<<(unsigned)((HW + 255) / 256), 256, 0, s>>>(pC, pT, order, K, HW, bg[0], bg[1], bg[2], image, T_out);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_merge_bwd(const float* pC, const float* pT, const int32_t* order, int K, int H, int W, const float bg[3],
                     const float* gI, const float* gT, float* dC, float* dT, cudaStream_t s) {
    int64_t HW = (int64_t)H * W;
    merge_bwd_kernel<<<(unsigned)((HW + 255) / 256), 256, 0, s>>>(pC, pT, order, K, HW, bg[0], bg[1], bg[2], gI, gT, dC,
                                                                  dT);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

}  // namespace rgs
