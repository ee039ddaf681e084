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
// Per-splat 2D gradients are reduced across the warp with shuffles, across the CTA in
// shared memory, and added to global memory with one vector reduction per float4.
#include <cuda_fp16.h>

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
// Instances of one splat (record id, first instance slot `base`), written by the calling
// warp; global tile indices start at tile_base.
__device__ __forceinline__ void emit_one(const ViewParams& vp, const TreeParams& tp, uint32_t id, uint32_t base,
                                         uint32_t tile_base, const ushort4* __restrict__ rect,
                                         const unsigned long long* __restrict__ mask, const float4* __restrict__ rec,
                                         const float* __restrict__ cull, const float2* __restrict__ chunk,
                                         uint32_t* __restrict__ ikey, uint32_t* __restrict__ ival, int lane) {
    const ushort4 r = rect[id];
    const unsigned long long m = mask[id];
    const float4 r0 = rec[3 * (size_t)id], r1 = rec[3 * (size_t)id + 1], r2 = rec[3 * (size_t)id + 2];
    const Footprint f = make_footprint(r0.x, r0.y, r1.x, r1.y, r1.z, r0.w, r1.w, vp);
    const int ty0 = r.y, rows = (int)r.w - (int)r.y + 1;
    const int nsub = __popcll(m);
    const int items = nsub * rows;
    for (int it0 = 0; it0 < items; it0 += 32) {
        const int it = it0 + lane;
        int c0 = 1, c1 = 0, ty = 0;
        uint32_t rank = 0;
        if (it < items) {
            int k;
            item_span(f, vp, tp, m, nsub, r2.w, ty0, rows, it, ty, k, c0, c1);
            rank = (uint32_t)vp.rank_of[k];
        }
        const uint32_t w = kept_tiles(cull, chunk, vp, ty, c0, c1, (int)rank, r2.w);
        uint32_t incl = w;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t pos = base + incl - w;
        const uint32_t first = tile_base + (uint32_t)(ty * vp.tiles_x);
        if (w && !cull) {
            for (int c = c0; c <= c1; ++c, ++pos) {
                ikey[pos] = ((first + (uint32_t)c) << vp.L) | rank;
                ival[pos] = id;
            }
        } else if (w) {
            const int nch = cull_nchunk(vp);
            for (int ch = c0 / kCullChunk; ch <= c1 / kCullChunk; ++ch) {
                const int lo = max(c0, ch * kCullChunk), hi = min(c1, ch * kCullChunk + kCullChunk - 1);
                const float2 mm = chunk[((size_t)ty * nch + ch) * vp.K + rank];
                if (r2.w > mm.y) continue;
                const bool all = r2.w <= mm.x;
                for (int c = lo; c <= hi; ++c) {
                    if (!all && !keep_tile(cull, vp, ty, c, (int)rank, r2.w)) continue;
                    ikey[pos] = ((first + (uint32_t)c) << vp.L) | rank;
                    ival[pos] = id;
                    ++pos;
                }
            }
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
}

__global__ void __launch_bounds__(256)
emit_kernel(ViewParams vp, TreeParams tp, const uint32_t* __restrict__ sorted_ids, int64_t n_vis,
            const uint32_t* __restrict__ ioff, const ushort4* __restrict__ rect,
            const unsigned long long* __restrict__ mask, const float4* __restrict__ rec, const float* __restrict__ cull,
            const float2* __restrict__ chunk, uint32_t* __restrict__ ikey, uint32_t* __restrict__ ival) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < n_vis; p += nwarps)
        emit_one(vp, tp, sorted_ids[p], ioff[p], 0u, rect, mask, rec, cull, chunk, ikey, ival, lane);
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

// Batch emission: sorted ids are slot * N + i, so each warp takes its splat's view from
// the block's shared copy of the slot table.
__global__ void __launch_bounds__(256)
emit_batch_kernel(const BatchSlot* __restrict__ slots, const BatchHeader* __restrict__ hdr, TreeParams tp,
                  const uint32_t* __restrict__ sorted_ids, int64_t n_cap, int64_t N,
                  const unsigned long long* __restrict__ counters, const uint32_t* __restrict__ ioff,
                  const ushort4* __restrict__ rect, const unsigned long long* __restrict__ mask,
                  const float4* __restrict__ rec, uint32_t* __restrict__ ikey, uint32_t* __restrict__ ival) {
    if (counters[2]) return;   // overflow: the batch is discarded
    __shared__ ViewParams svp[kMaxSlots];
    __shared__ uint32_t sbase[kMaxSlots];
    const int S = hdr->S;
    if ((int)threadIdx.x < S) sbase[threadIdx.x] = hdr->tile_base[threadIdx.x];
    load_batch_views(slots, S, svp);
    const unsigned long long nv = counters[1];
    const int64_t n = nv < (unsigned long long)n_cap ? (int64_t)nv : n_cap;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < n; p += nwarps) {
        const uint32_t id = sorted_ids[p];
        const int slot = (int)(id / (uint64_t)N);
        emit_one(svp[slot], tp, id, ioff[p], sbase[slot], rect, mask, rec, nullptr, nullptr, ikey, ival, lane);
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
    float lo = __int_as_float(0x7f800000), hi = -lo;
    for (int c = ch * kCullChunk; c < min(vp.tiles_x, (ch + 1) * kCullChunk); ++c) {
        const float d = cull[((size_t)ty * vp.tiles_x + c) * vp.K + rank];
        lo = fminf(lo, d);
        hi = fmaxf(hi, d);
    }
    chunk[i] = make_float2(lo, hi);
}

__global__ void ranges_kernel(const uint32_t* __restrict__ keys, int64_t n, uint2* __restrict__ ranges) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t k = keys[j];
    if (j == 0 || keys[j - 1] != k) ranges[k].x = (uint32_t)j;
    if (j == n - 1 || keys[j + 1] != k) ranges[k].y = (uint32_t)(j + 1);
}

__global__ void ranges_dev_kernel(const uint32_t* __restrict__ keys, const unsigned long long* __restrict__ n_dev,
                                  int64_t cap, uint2* __restrict__ ranges) {
    const unsigned long long nv = *n_dev;
    const int64_t n = nv < (unsigned long long)cap ? (int64_t)nv : cap;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[j];
        if (j == 0 || keys[j - 1] != k) ranges[k].x = (uint32_t)j;
        if (j == n - 1 || keys[j + 1] != k) ranges[k].y = (uint32_t)(j + 1);
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

struct StagedRec {   // tile-relative record in shared memory (3 x float4)
    float4 a;        // mx, my, alpha, rho2 (sign: straddles several subsets)
    float4 b;        // l11, l12, l22, z
    float4 c;        // r, g, b, (splat id as bits)
};

// Bit w set: the footprint can touch warp w's 8x4 block (one span per 4-row band); for a
// splat held by several subsets the span is also clipped to the current subset (Eq. 6).
__device__ __forceinline__ uint32_t block_mask(const StagedRec& r, const ViewParams& vp, const LeafPath& lp, float x0t,
                                               float y0t) {
    const Footprint f = make_footprint(r.a.x, r.a.y, r.b.x, r.b.y, r.b.z, r.a.z, r.a.w, vp);
    const bool straddles = r.a.w < 0.f;
    SubsetClip clip;
    if (straddles) make_clip(vp, lp, vp.L, r.b.w, clip);
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

__device__ __forceinline__ StagedRec stage_record(const float4* __restrict__ rec, uint32_t id, float x0, float y0) {
    float4 r0 = rec[3 * (size_t)id], r1 = rec[3 * (size_t)id + 1], r2 = rec[3 * (size_t)id + 2];
    uint32_t lo_bits = __float_as_uint(r0.z);
    __half2 lo = *reinterpret_cast<__half2*>(&lo_bits);
    float2 lof = __half22float2(lo);
    StagedRec s;
    s.a = make_float4(__fadd_rn(__fsub_rn(r0.x, x0), lof.x), __fadd_rn(__fsub_rn(r0.y, y0), lof.y), r0.w, r1.w);
    s.b = make_float4(r1.x, r1.y, r1.z, r2.w);
    s.c = make_float4(r2.x, r2.y, r2.z, __uint_as_float(id));
    return s;
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
// One tile of the view: `ranges` and `tile_depth` point at the tile's K entries (view
// rank order); pC/pT (partial maps) and tile_depth may be null.  The whole block calls it.
template <bool kCount>
__device__ __forceinline__ void blend_fwd_tile(const ViewParams& vp, const TreeParams& tp, int tile,
                                               const uint2* __restrict__ ranges, const uint32_t* __restrict__ ival,
                                               const float4* __restrict__ rec, float* __restrict__ pC,
                                               float* __restrict__ pT, float* __restrict__ image,
                                               float* __restrict__ Tfin, float* __restrict__ tile_depth,
                                               unsigned long long* __restrict__ pairs) {
    __shared__ StagedRec srec[kBlendThreads];
    __shared__ uint32_t smask[kBlendThreads];
    __shared__ float4 splane[kBlendThreads][kMaxCutPlanes];
    __shared__ LeafPath lp;
    __shared__ uint32_t sused[kBlendThreads];
    uint32_t n_eval = 0, n_contrib = 0, n_d2 = 0, n_ball = 0, n_leaf = 0, n_strad = 0, n_staged = 0, n_used = 0;
    const int tyi = tile / vp.tiles_x, txi = tile - tyi * vp.tiles_x;
    int lx, ly;
    thread_pixel(threadIdx.x, lx, ly);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px = txi * kTile + lx, py = tyi * kTile + ly;
    const bool inside = px < vp.W && py < vp.H;
    const float x0 = (float)(txi * kTile), y0 = (float)(tyi * kTile);
    const float pcx = lx + 0.5f, pcy = ly + 0.5f;
    const float Xc = (float)px + 0.5f, Yc = (float)py + 0.5f;   // absolute pixel centre (Eq. 6 tests)
    const float tm2 = vp.trunc_mult * vp.trunc_mult;
    const size_t HW = (size_t)vp.W * vp.H;
    const size_t pix = (size_t)py * vp.W + px;
    float img0 = 0.f, img1 = 0.f, img2 = 0.f, Pm = 1.f;

    for (int r = 0; r < vp.K; ++r) {
        const int k = vp.order[r];
        if (threadIdx.x == 0) leaf_path(tp, k, lp);   // read only after the next barrier
        const uint2 rg = ranges[r];
        float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
        bool done = !inside;
        float zsat = __int_as_float(0x7f800000);   // +inf: the subset never saturated the tile
        for (uint32_t b0 = rg.x; b0 < rg.y; b0 += kBlendThreads) {
            const int nb = (int)min((uint32_t)kBlendThreads, rg.y - b0);
            __syncthreads();
            if ((int)threadIdx.x < nb) {
                StagedRec sr = stage_record(rec, ival[b0 + threadIdx.x], x0, y0);
                uint32_t msk = block_mask(sr, vp, lp, x0, y0);
                if (sr.a.w < 0.f && msk) {
                    const int nc = classify_planes(vp, lp, sr.b.w, x0 + 0.5f, y0 + 0.5f, splane[threadIdx.x]);
                    if (nc < 0) msk = 0;                        // no pixel of the tile is in this subset
                    else if (nc == 0) sr.a.w = -sr.a.w;         // every pixel is: no per-pixel test
                    else msk |= (uint32_t)nc << 8;
                }
                srec[threadIdx.x] = sr;
                smask[threadIdx.x] = msk;
                if (kCount) {
                    sused[threadIdx.x] = 0;
                    ++n_staged;
                }
            }
            __syncthreads();
            for (int c0 = 0; c0 < nb && !__all_sync(0xffffffffu, done); c0 += 32) {
                unsigned bits = __ballot_sync(0xffffffffu, c0 + lane < nb && ((smask[c0 + lane] >> warp) & 1u));
                while (bits) {
                    const int j = c0 + __ffs(bits) - 1;
                    bits &= bits - 1;
                    // Branch-free body: a pair that fails a test (or a pixel already done)
                    // gets sigma = 0, which leaves C and T unchanged.  The backward repeats
                    // this arithmetic exactly.
                    const float4 A = srec[j].a;
                    const float4 B = srec[j].b;
                    const float dx = pcx - A.x, dy = pcy - A.y;
                    const float u1 = fmaf(B.x, dx, B.y * dy), u2 = B.z * dy;
                    const float d2 = fmaf(u1, u1, u2 * u2);
                    const float bx = dx * vp.ifx, by = dy * vp.ify;
                    const bool in_ell = d2 <= tm2, in_ball = fmaf(bx, bx, by * by) <= fabsf(A.w);
                    bool ok = !done && in_ell && in_ball;
                    bool in_sub = true;
                    if (A.w < 0.f) {   // uniform across the warp: one record
                        in_sub = in_subset(splane[j], (int)((smask[j] >> 8) & 7u), vp, lp, B.w, Xc, Yc);
                        ok = ok && in_sub;
                    }
                    const float G = ex2_approx(d2 * kNegHalfLog2e);
                    float sig = fminf(A.z * G, vp.alpha_max);
                    ok = ok && sig >= vp.alpha_min;
                    if (kCount && !done) {
                        ++n_eval;
                        n_strad += A.w < 0.f;
                        n_d2 += !in_ell;
                        n_ball += in_ell && !in_ball;
                        n_leaf += in_ell && in_ball && !in_sub;
                        n_contrib += ok;
                        if (ok) sused[j] = 1;
                    }
                    sig = ok ? sig : 0.f;
                    const float4 Cc = srec[j].c;
                    const float w = sig * T;
                    C0 = fmaf(Cc.x, w, C0);
                    C1 = fmaf(Cc.y, w, C1);
                    C2 = fmaf(Cc.z, w, C2);
                    T = fmaf(-sig, T, T);
                    done = done || T < vp.eps_T;
                }
            }
            if (kCount) {
                __syncthreads();
                if ((int)threadIdx.x < nb) n_used += sused[threadIdx.x];
            }
            if (__syncthreads_count(done) == kBlendThreads) {
                zsat = srec[nb - 1].b.w;   // depth of the last instance staged
                break;
            }
        }
        if (tile_depth && threadIdx.x == 0) tile_depth[r] = zsat;
        if (inside) {
            if (pC) {
                pC[((size_t)k * 3 + 0) * HW + pix] = C0;
                pC[((size_t)k * 3 + 1) * HW + pix] = C1;
                pC[((size_t)k * 3 + 2) * HW + pix] = C2;
                pT[(size_t)k * HW + pix] = T;
            }
            img0 = fmaf(C0, Pm, img0);
            img1 = fmaf(C1, Pm, img1);
            img2 = fmaf(C2, Pm, img2);
            Pm *= T;
        }
    }
    if (inside && image) {
        image[0 * HW + pix] = fmaf(vp.bg[0], Pm, img0);
        image[1 * HW + pix] = fmaf(vp.bg[1], Pm, img1);
        image[2 * HW + pix] = fmaf(vp.bg[2], Pm, img2);
        if (Tfin) Tfin[pix] = Pm;
    }
    if (kCount) {
        count_pairs(pairs, n_eval, n_contrib);
        count_add(pairs + 4, n_d2);
        count_add(pairs + 5, n_ball);
        count_add(pairs + 6, n_leaf);
        count_add(pairs + 7, n_strad);
        count_add(pairs + 8, n_staged);
        count_add(pairs + 9, n_used);
    }
}

template <bool kCount>
__global__ void __launch_bounds__(kBlendThreads, RGS_BLEND_MIN_BLOCKS)
blend_fwd_kernel(ViewParams vp, TreeParams tp, const uint2* __restrict__ ranges, const uint32_t* __restrict__ ival,
                 const float4* __restrict__ rec, float* __restrict__ pC, float* __restrict__ pT,
                 float* __restrict__ image, float* __restrict__ Tfin, float* __restrict__ tile_depth,
                 unsigned long long* __restrict__ pairs) {
    const int tile = blockIdx.x;
    blend_fwd_tile<kCount>(vp, tp, tile, ranges + (size_t)tile * vp.K, ival, rec, pC, pT, image, Tfin,
                           tile_depth ? tile_depth + (size_t)tile * vp.K : nullptr, pairs);
}

// Persistent forward blend over the global tiles of a batch: each block takes the next
// tile from a device counter until all are done; a tile belongs to the last request
// whose tile_base it reaches.  The request's view is kept in shared memory while
// consecutive tiles stay in one request.
__global__ void __launch_bounds__(kBlendThreads, RGS_BLEND_MIN_BLOCKS)
blend_batch_kernel(const BatchSlot* __restrict__ slots, const BatchHeader* __restrict__ hdr, TreeParams tp,
                   const uint2* __restrict__ ranges, const uint32_t* __restrict__ ival, const float4* __restrict__ rec,
                   unsigned long long* __restrict__ counters) {
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
        blend_fwd_tile<false>(svp, tp, (int)(t - hdr->tile_base[slot]), ranges + (size_t)t * svp.K, ival, rec,
                              nullptr, nullptr, slots[slot].image, nullptr, nullptr, nullptr);
        __syncthreads();   // s_tile is rewritten by the next claim
    }
}

// ------------------------------------------------------------------ blend backward
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums v[0..15] over the 32 lanes of a warp with 16 shuffles (reduce-scatter by halving):
// at each step a lane keeps one half of its values, sends the other half to its partner
// and adds what it receives.  Returns the total of value index (lane >> 1) & 15; both
// lanes of each pair hold it.
__device__ __forceinline__ float warp_reduce16(float (&v)[16], int lane) {
#pragma unroll
    for (int h = 8, off = 16; h >= 1; h >>= 1, off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const float send = upper ? v[k] : v[k + h];
            const float keep = upper ? v[k + h] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ void red_add_v4(float4* addr, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

// dynamic shared memory: s_behind [K][256] floats
template <bool kCount>
__global__ void __launch_bounds__(kBlendThreads, RGS_BLEND_MIN_BLOCKS)
blend_bwd_kernel(ViewParams vp, TreeParams tp, const uint2* __restrict__ ranges, const uint32_t* __restrict__ ival,
                 const float4* __restrict__ rec, const float* __restrict__ pC, const float* __restrict__ pT,
                 const float* __restrict__ gI, float4* __restrict__ g2d, unsigned long long* __restrict__ pairs) {
    extern __shared__ float s_behind[];
    uint32_t n_eval = 0, n_contrib = 0;
    __shared__ StagedRec srec[kBlendThreads];
    __shared__ uint32_t smask[kBlendThreads];
    __shared__ float4 splane[kBlendThreads][kMaxCutPlanes];
    __shared__ float sacc[kBlendThreads][9];
    __shared__ LeafPath lp;
    const int tile = blockIdx.x;
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
    const float tm2 = vp.trunc_mult * vp.trunc_mult;
    const size_t HW = (size_t)vp.W * vp.H;
    const size_t pix = inside ? (size_t)py * vp.W + px : 0;

    for (int i = threadIdx.x; i < kBlendThreads * 9; i += kBlendThreads) (&sacc[0][0])[i] = 0.f;

    // adjoint of Eq. 5: <g, S_r> for every rank, back to front
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (inside) {
        g0 = gI[0 * HW + pix];
        g1 = gI[1 * HW + pix];
        g2 = gI[2 * HW + pix];
    }
    {
        float behind = g0 * vp.bg[0] + g1 * vp.bg[1] + g2 * vp.bg[2];
        for (int r = vp.K - 1; r >= 0; --r) {
            s_behind[r * kBlendThreads + threadIdx.x] = behind;
            if (inside) {
                const int k = vp.order[r];
                float c0 = pC[((size_t)k * 3 + 0) * HW + pix], c1 = pC[((size_t)k * 3 + 1) * HW + pix],
                      c2 = pC[((size_t)k * 3 + 2) * HW + pix], t = pT[(size_t)k * HW + pix];
                behind = fmaf(t, behind, g0 * c0 + g1 * c1 + g2 * c2);
            }
        }
    }
    float Pm = 1.f;
    for (int r = 0; r < vp.K; ++r) {
        const int k = vp.order[r];
        float Ck0 = 0.f, Ck1 = 0.f, Ck2 = 0.f, Tk = 1.f;
        if (inside) {
            Ck0 = pC[((size_t)k * 3 + 0) * HW + pix];
            Ck1 = pC[((size_t)k * 3 + 1) * HW + pix];
            Ck2 = pC[((size_t)k * 3 + 2) * HW + pix];
            Tk = pT[(size_t)k * HW + pix];
        }
        const float gC0 = g0 * Pm, gC1 = g1 * Pm, gC2 = g2 * Pm;
        const float gT = Pm * s_behind[r * kBlendThreads + threadIdx.x];
        const float q = gC0 * Ck0 + gC1 * Ck1 + gC2 * Ck2 + gT * Tk;
        Pm *= Tk;
        if (threadIdx.x == 0) leaf_path(tp, k, lp);   // read only after the next barrier
        const uint2 rg = ranges[(size_t)tile * vp.K + r];
        bool active = inside && (gC0 != 0.f || gC1 != 0.f || gC2 != 0.f || gT != 0.f);
        if (__syncthreads_count(active) == 0) continue;
        bool done = !active;
        float T = 1.f, acc = 0.f;   // acc = <gC, A_i>
        for (uint32_t b0 = rg.x; b0 < rg.y; b0 += kBlendThreads) {
            const int nb = (int)min((uint32_t)kBlendThreads, rg.y - b0);
            __syncthreads();
            if ((int)threadIdx.x < nb) {
                StagedRec sr = stage_record(rec, ival[b0 + threadIdx.x], x0, y0);
                uint32_t msk = block_mask(sr, vp, lp, x0, y0);
                if (sr.a.w < 0.f && msk) {
                    const int nc = classify_planes(vp, lp, sr.b.w, x0 + 0.5f, y0 + 0.5f, splane[threadIdx.x]);
                    if (nc < 0) msk = 0;                        // no pixel of the tile is in this subset
                    else if (nc == 0) sr.a.w = -sr.a.w;         // every pixel is: no per-pixel test
                    else msk |= (uint32_t)nc << 8;
                }
                srec[threadIdx.x] = sr;
                smask[threadIdx.x] = msk;
            }
            __syncthreads();
            for (int c0 = 0; c0 < nb && !__all_sync(0xffffffffu, done); c0 += 32) {
                unsigned bits = __ballot_sync(0xffffffffu, c0 + lane < nb && ((smask[c0 + lane] >> warp) & 1u));
                while (bits) {
                    const int j = c0 + __ffs(bits) - 1;
                    bits &= bits - 1;
                    // the forward's arithmetic, then the adjoint of the pair with the same
                    // predicate (a pair that fails gets sigma = 0 and zero gradients)
                    const float4 A = srec[j].a;
                    const float4 B = srec[j].b;
                    const float dx = pcx - A.x, dy = pcy - A.y;
                    const float u1 = fmaf(B.x, dx, B.y * dy), u2 = B.z * dy;
                    const float d2 = fmaf(u1, u1, u2 * u2);
                    const float bx = dx * vp.ifx, by = dy * vp.ify;
                    bool ok = !done && d2 <= tm2 && fmaf(bx, bx, by * by) <= fabsf(A.w);
                    if (A.w < 0.f)   // uniform across the warp: one record
                        ok = ok && in_subset(splane[j], (int)((smask[j] >> 8) & 7u), vp, lp, B.w, Xc, Yc);
                    const float G = ex2_approx(d2 * kNegHalfLog2e);
                    const float raw = A.z * G;
                    float sig = fminf(raw, vp.alpha_max);
                    ok = ok && sig >= vp.alpha_min;
                    if (kCount && !done) {
                        ++n_eval;
                        n_contrib += ok;
                    }
                    sig = ok ? sig : 0.f;
                    const float4 Cc = srec[j].c;
                    const float w = sig * T;
                    const float grgb = gC0 * Cc.x + gC1 * Cc.y + gC2 * Cc.z;
                    acc = fmaf(w, grgb, acc);
                    const float dsig = T * grgb - __fdividef(q - acc, 1.f - sig);
                    const float gr0 = gC0 * w, gr1 = gC1 * w, gr2 = gC2 * w;
                    const float ds = (ok && raw < vp.alpha_max) ? dsig : 0.f;
                    const float gal = ds * G;
                    const float gd2 = -0.5f * sig * ds;
                    const float ga = gd2 * dx * dx, gb = gd2 * 2.f * dx * dy, gc = gd2 * dy * dy;
                    // d(d2)/d(mean) = -2 Q delta, Q delta = L^T (u1, u2)
                    const float gmx = -2.f * gd2 * (B.x * u1);
                    const float gmy = -2.f * gd2 * fmaf(B.y, u1, B.z * u2);
                    T = fmaf(-sig, T, T);
                    done = done || T < vp.eps_T;
                    const bool contrib = ok;
                    if (__any_sync(0xffffffffu, contrib)) {
                        float v[16] = {gmx, gmy, ga, gb, gc, gal, gr0, gr1, gr2, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                        const float tot = warp_reduce16(v, lane);
                        const int vi = (lane >> 1) & 15;
                        if ((lane & 1) == 0 && vi < 9) atomicAdd(&sacc[j][vi], tot);
                    }
                }
            }
            __syncthreads();
            if ((int)threadIdx.x < nb) {
                float* a = sacc[threadIdx.x];
                bool nz = false;
                for (int t = 0; t < 9; ++t) nz |= a[t] != 0.f;
                if (nz) {
                    const uint32_t id = __float_as_uint(srec[threadIdx.x].c.w);
                    float4* dst = g2d + 3 * (size_t)id;
                    red_add_v4(dst, make_float4(a[0], a[1], a[2], a[3]));
                    red_add_v4(dst + 1, make_float4(a[4], a[5], a[6], a[7]));
                    red_add_v4(dst + 2, make_float4(a[8], 0.f, 0.f, 0.f));
                    for (int t = 0; t < 9; ++t) a[t] = 0.f;
                }
            }
            if (__syncthreads_count(done) == kBlendThreads) break;
        }
    }
    if (kCount) count_pairs(pairs + 2, n_eval, n_contrib);
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
    const int64_t want = (n_vis + 7) / 8;          // one warp per splat
    unsigned grid = (unsigned)(want < (1 << 20) ? want : (1 << 20));
    emit_kernel<<<grid, 256, 0, s>>>(vp, tp, sorted_ids, n_vis, b.ioff, b.rect, b.mask, b.rec, b.cull, b.cull_chunk, b.ikey, b.ival);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_cull_chunks(const ViewParams& vp, const float* cull, float2* chunk, cudaStream_t s) {
    const int64_t total = (int64_t)vp.tiles_y * ((vp.tiles_x + kCullChunk - 1) / kCullChunk) * vp.K;
    cull_chunk_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(vp, cull, chunk);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_ranges(const uint32_t* keys, int64_t n, uint2* ranges, int64_t n_ranges, cudaStream_t s) {
    RGS_CUDA_TRY(cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_ranges, s));
    if (n <= 0) return RGS_OK;
    ranges_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, ranges);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_blend_fwd(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* ival,
                     float* partial_C, float* partial_T, float* image, float* T_final, float* tile_depth,
                     cudaStream_t s) {
    unsigned grid = (unsigned)(vp.tiles_x * vp.tiles_y);
    unsigned long long* pairs = prof_pair_counters();
    if (pairs)
        blend_fwd_kernel<true><<<grid, kBlendThreads, 0, s>>>(vp, tp, b.ranges, ival, b.rec, partial_C, partial_T, image,
                                                              T_final, tile_depth, pairs);
    else
        blend_fwd_kernel<false><<<grid, kBlendThreads, 0, s>>>(vp, tp, b.ranges, ival, b.rec, partial_C, partial_T,
                                                               image, T_final, tile_depth, nullptr);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_emit_batch(const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp, const RasterBuffers& b,
                      const uint32_t* sorted_ids, int64_t n_cap, int64_t N, const unsigned long long* counters,
                      cudaStream_t s) {
    emit_batch_kernel<<<152 * 8, 256, 0, s>>>(slots, hdr, tp, sorted_ids, n_cap, N, counters, b.ioff, b.rect, b.mask,
                                              b.rec, b.ikey, b.ival);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_ranges_dev(const uint32_t* keys, const unsigned long long* n_dev, int64_t cap, uint2* ranges,
                      cudaStream_t s) {
    ranges_dev_kernel<<<152 * 8, 256, 0, s>>>(keys, n_dev, cap, ranges);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_blend_batch(const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp, const uint2* ranges,
                       const uint32_t* ival, const float4* rec, unsigned long long* counters, cudaStream_t s) {
    int dev = 0, sms = 0;
    RGS_CUDA_TRY(cudaGetDevice(&dev));
    RGS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    blend_batch_kernel<<<(unsigned)(sms * RGS_BLEND_MIN_BLOCKS), kBlendThreads, 0, s>>>(slots, hdr, tp, ranges, ival,
                                                                                      rec, counters);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_blend_bwd(const ViewParams& vp, const TreeParams& tp, const RasterBuffers& b, const uint32_t* ival,
                     const float* partial_C, const float* partial_T, const float* dL_dimage, cudaStream_t s) {
    unsigned grid = (unsigned)(vp.tiles_x * vp.tiles_y);
    size_t smem = sizeof(float) * (size_t)vp.K * kBlendThreads;
    static bool attr_set = false;
    if (!attr_set) {
        RGS_CUDA_TRY(cudaFuncSetAttribute(blend_bwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        RGS_CUDA_TRY(cudaFuncSetAttribute(blend_bwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        attr_set = true;
    }
    unsigned long long* pairs = prof_pair_counters();
    if (pairs)
        blend_bwd_kernel<true><<<grid, kBlendThreads, smem, s>>>(vp, tp, b.ranges, ival, b.rec, partial_C, partial_T,
                                                                 dL_dimage, b.g2d, pairs);
    else
        blend_bwd_kernel<false><<<grid, kBlendThreads, smem, s>>>(vp, tp, b.ranges, ival, b.rec, partial_C, partial_T,
                                                                  dL_dimage, b.g2d, nullptr);
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
