// Device-wide exclusive scan and stable LSD radix sort of (uint32 key, uint32 value)
// pairs.  They carry the tile binning ("tile-binned") and the per-subset depth order
// ("depth-sorted", Sec. 3.1-3.2) of the render, and the median splits of the KD tree.
//
// Scan: reduce-then-scan over 4096-element tiles, recursive on the tile sums.
// Radix sort: per 8-bit digit an upsweep (per-tile digit histogram), a scan of the
// digit-major histogram, and a downsweep that ranks keys stably inside the tile with
// warp-level match/popc, stages the tile in shared memory in digit order and writes runs
// of equal digits to their global positions.
#include <cstdio>

#include "rgs_internal.cuh"

namespace rgs {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;   // 4096

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;   // 2048

__device__ __forceinline__ uint32_t load_item(const uint32_t* in, const uint32_t* gather, int64_t i, int mode) {
    uint32_t v = mode == 2 ? in[gather[i]] : in[i];
    return mode == 1 ? (v != 0u) : v;
}

// Sum of one tile (block) of the input.
__global__ void __launch_bounds__(kScanThreads)
scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n, int mode, const uint32_t* __restrict__ gather,
                   uint32_t* __restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t acc = 0;
    for (int j = 0; j < kScanItems; ++j) {
        int64_t i = base + (int64_t)j * kScanThreads + threadIdx.x;
        if (i < n) acc += load_item(in, gather, i, mode);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ uint32_t ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// Exclusive scan of the tile [base, base + kScanTile) of the input plus `offset`; returns
// the tile's total.  Items are loaded coalesced into shared memory (padded against bank
// conflicts), each thread scans 16 consecutive items, and the thread totals are scanned
// across the block.  In-place use (in == out) is safe: the tile is read before it is written.
__device__ __forceinline__ uint32_t scan_tile_body(const uint32_t* in, uint32_t* out, int64_t n, int mode,
                                                   const uint32_t* __restrict__ gather, int64_t base,
                                                   uint32_t offset) {
    __shared__ uint32_t sm[kScanTile + kScanTile / 32];
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    auto pad = [](int i) { return i + (i >> 5); };
    for (int j = 0; j < kScanItems; ++j) {
        int li = j * kScanThreads + threadIdx.x;
        int64_t i = base + li;
        sm[pad(li)] = i < n ? load_item(in, gather, i, mode) : 0u;
    }
    __syncthreads();
    uint32_t v[kScanItems];
    uint32_t tsum = 0;
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = sm[pad(threadIdx.x * kScanItems + j)];
        tsum += v[j];
    }
    // inclusive warp scan of the thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = tsum;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint32_t wbase = offset, total = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        if (w < warp) wbase += warp_tot[w];
        total += warp_tot[w];
    }
    uint32_t run = wbase + incl - tsum;
    for (int j = 0; j < kScanItems; ++j) {
        uint32_t x = v[j];
        sm[pad(threadIdx.x * kScanItems + j)] = run;
        run += x;
    }
    __syncthreads();
    for (int j = 0; j < kScanItems; ++j) {
        int li = j * kScanThreads + threadIdx.x;
        int64_t i = base + li;
        if (i < n) out[i] = sm[pad(li)];
    }
    __syncthreads();   // the shared tile is reused by the caller's next tile
    return total;
}

__global__ void __launch_bounds__(kScanThreads)
scan_tile_kernel(const uint32_t* in, uint32_t* out, int64_t n, int mode, const uint32_t* __restrict__ gather,
                 const uint32_t* __restrict__ tile_offsets) {
    scan_tile_body(in, out, n, mode, gather, (int64_t)blockIdx.x * kScanTile,
                   tile_offsets ? tile_offsets[blockIdx.x] : 0u);
}

// A block of the host-counted passes owns kBlockTiles consecutive sort tiles, so the
// digit-major count table (read and written with a stride of the block count) stays small.
constexpr int kBlockTiles = 8;
constexpr int kBlockItems = kSortTile * kBlockTiles;   // 16384

// Adds the digits of keys [lo, hi) to the shared histogram: a thread takes 8 consecutive
// keys per round (two 16-byte loads when `vec` and lo is a multiple of 8) and adds each
// run of equal digits with one shared atomic (the later passes see keys already ordered
// by their low digits, whose high digits repeat).  The whole block calls it.
template <int kThreads = kSortThreads, uint32_t kMask = kRadix - 1>
__device__ __forceinline__ void hist_runs(const uint32_t* __restrict__ keys, int64_t lo, int64_t hi, int shift, bool vec,
                                          uint32_t* hist) {
    for (int64_t b = lo; b < hi; b += kThreads * 8) {   // uniform trip count across the block
        const int64_t i0 = b + (int64_t)threadIdx.x * 8;
        uint32_t k[8];
        if (vec && i0 + 8 <= hi) {
            const uint4 x = *reinterpret_cast<const uint4*>(keys + i0);
            const uint4 y = *reinterpret_cast<const uint4*>(keys + i0 + 4);
            k[0] = x.x; k[1] = x.y; k[2] = x.z; k[3] = x.w; k[4] = y.x; k[5] = y.y; k[6] = y.z; k[7] = y.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) k[j] = i0 + j < hi ? keys[i0 + j] : 0u;
        }
        const int m = hi - i0 < 8 ? (int)(hi - i0) : 8;   // may be <= 0 past the end
        if (m > 0) {
            uint32_t cur = (k[0] >> shift) & kMask, run = 1;
#pragma unroll
            for (int j = 1; j < 8; ++j) {
                if (j >= m) break;
                const uint32_t d = (k[j] >> shift) & kMask;
                if (d != cur) {
                    atomicAdd(&hist[cur], run);
                    cur = d;
                    run = 0;
                }
                ++run;
            }
            atomicAdd(&hist[cur], run);
        }
    }
}

// Histogram of one 8-bit digit over the block's range, written digit-major:
// counts[d * nblocks + b].
__global__ void __launch_bounds__(kSortThreads, 4)
radix_upsweep_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ counts,
                     uint32_t nblocks, bool vec) {
    __shared__ uint32_t hist[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) hist[d] = 0;
    __syncthreads();
    const int64_t lo = (int64_t)blockIdx.x * kBlockItems;
    hist_runs(keys, lo, min(n, lo + kBlockItems), shift, vec, hist);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) counts[(int64_t)d * nblocks + blockIdx.x] = hist[d];
}

// Stable scatter of the tile [base, base + count) (count <= kSortTile) by one digit.
// Warp w owns tile items [w*256, (w+1)*256) and walks them in 8 rounds of 32 lanes, so
// (round, lane) order is the input order; a per-warp digit counter plus the rank among
// equal digits of the round gives each key's rank within its warp, the per-digit scan
// over warps gives its rank within the tile.  goff[d] (shared) is where the tile's first
// key of digit d goes; on return it has advanced past the tile's keys of digit d.
// This thread's items of the tile [base, base + count) in the order radix_rank_scatter
// expects them.
__device__ __forceinline__ void radix_tile_load(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                int64_t base, int count, uint32_t (&key)[kSortItems],
                                                uint32_t (&val)[kSortItems]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int li = warp * (kSortItems * 32) + r * 32 + lane;
        const bool ok = li < count;
        key[r] = ok ? kin[base + li] : 0u;
        val[r] = ok ? vin[base + li] : 0u;
    }
}

__device__ __forceinline__ void radix_rank_scatter(const uint32_t (&key)[kSortItems], const uint32_t (&val)[kSortItems],
                                                   uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                   int count, int shift, uint32_t* goff) {
    __shared__ uint32_t whist[kSortWarps][kRadix];
    __shared__ uint32_t dstart[kRadix];
    __shared__ uint32_t dtot[kRadix];
    __shared__ uint32_t wsum[kSortWarps];
    __shared__ uint32_t skeys[kSortTile];
    __shared__ uint32_t svals[kSortTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&whist[0][0])[i] = 0;
    __syncthreads();

    uint32_t rank[kSortItems];
    int dig[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int li = warp * (kSortItems * 32) + r * 32 + lane;
        dig[r] = li < count ? (int)((key[r] >> shift) & (kRadix - 1)) : kRadix;
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        unsigned peers = __match_any_sync(0xffffffffu, dig[r]);
        unsigned lower = peers & ((1u << lane) - 1u);
        uint32_t prior = dig[r] < kRadix ? whist[warp][dig[r]] : 0u;
        rank[r] = prior + (uint32_t)__popc(lower);
        __syncwarp();
        if (dig[r] < kRadix && lower == 0u) whist[warp][dig[r]] = prior + (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            uint32_t c = whist[w][d];
            whist[w][d] = run;
            run += c;
        }
        dtot[d] = run;
    }
    __syncthreads();
    // exclusive scan of the digit totals (kRadix == kSortThreads: one per thread)
    {
        uint32_t x = dtot[threadIdx.x];
        uint32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t b = 0;
        for (int w = 0; w < warp; ++w) b += wsum[w];
        dstart[threadIdx.x] = b + incl - x;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (dig[r] < kRadix) {
            uint32_t pos = dstart[dig[r]] + whist[warp][dig[r]] + rank[r];
            skeys[pos] = key[r];
            svals[pos] = val[r];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += kSortThreads) {
        uint32_t k = skeys[i];
        int d = (int)((k >> shift) & (kRadix - 1));
        uint32_t o = goff[d] + (uint32_t)i - dstart[d];
        kout[o] = k;
        vout[o] = svals[i];
    }
    __syncthreads();
    goff[threadIdx.x] += dtot[threadIdx.x];
    __syncthreads();
}

__device__ __forceinline__ void radix_tile_body(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                int64_t base, int count, int shift, uint32_t* goff) {
    uint32_t key[kSortItems], val[kSortItems];
    radix_tile_load(kin, vin, base, count, key, val);
    radix_rank_scatter(key, val, kout, vout, count, shift, goff);
}

__global__ void __launch_bounds__(kSortThreads, 4)
radix_downsweep_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
                       uint32_t* __restrict__ vout, int64_t n, int shift, const uint32_t* __restrict__ offsets,
                       uint32_t nblocks) {
    __shared__ uint32_t goff[kRadix];
    goff[threadIdx.x] = offsets[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    const int64_t lo = (int64_t)blockIdx.x * kBlockItems;
    const int64_t hi = min(n, lo + kBlockItems);
    for (int64_t base = lo; base < hi; base += kSortTile) {   // tiles in order: stable
        const int64_t rem = hi - base;
        radix_tile_body(kin, vin, kout, vout, base, rem < kSortTile ? (int)rem : kSortTile, shift, goff);
    }
}

// ------------------------------------------------------------------ wide-digit passes
// Keys of 17 to 20 bits (the (tile, subset) keys of a 4K view) are sorted in two passes of
// up to 10 bits instead of three of 8: a third less traffic.  With 1024 digits a tile must
// be large for its runs of equal digits to fill whole sectors when they are written out,
// so a block of 512 threads ranks 8192 keys at a time (16 per thread), with 16-bit
// per-warp digit counters; the tile and the counters take 108 KB of shared memory, two
// blocks per SM.  Same structure as the 8-bit passes otherwise: per-block digit histograms
// written digit-major, one scan, a stable downsweep.
constexpr int kWideThreads = 512;
constexpr int kWideWarps = kWideThreads / 32;
constexpr int kWideItems = 16;
constexpr int kWideTile = kWideThreads * kWideItems;           // 8192
constexpr int kWideBlockTiles = 8;
constexpr int kWideBlockItems = kWideTile * kWideBlockTiles;   // 65536
constexpr int kWideMaxBits = 10;

// Blocks of the device-counted wide passes (two per SM).
constexpr int kWideChunks = 304;

// The keys block b owns: with n_dev, the b-th of nblocks contiguous chunks of whole
// tiles of the first min(*n_dev, n) keys; without, [b * kWideBlockItems, +kWideBlockItems).
__device__ __forceinline__ void wide_range(int64_t n, const unsigned long long* n_dev, uint32_t nblocks, int64_t& lo,
                                           int64_t& hi) {
    if (n_dev) {
        const unsigned long long v = *n_dev;
        const int64_t m = v < (unsigned long long)n ? (int64_t)v : n;
        const int64_t tiles = (m + kWideTile - 1) / kWideTile;
        const int64_t per = (tiles + nblocks - 1) / nblocks;
        lo = min(m, (int64_t)blockIdx.x * per * kWideTile);
        hi = min(m, lo + per * kWideTile);
    } else {
        lo = (int64_t)blockIdx.x * kWideBlockItems;
        hi = min(n, lo + kWideBlockItems);
    }
}

template <int kBits>
struct WideSmem {
    static constexpr int kBins = 1 << kBits;
    uint16_t whist[kWideWarps][kBins];   // per-warp digit counts, then each (warp, digit)'s first tile slot
    uint32_t skeys[kWideTile];
    uint32_t svals[kWideTile];
    uint32_t dtot[kBins];                // the tile's digit totals
    uint32_t goff[kBins];                // where the block's next key of each digit goes
    uint32_t gbase[kBins];               // goff - (first tile slot of the digit), for the write-out
    uint32_t wsum[kWideWarps];
};

template <int kBits>
__global__ void __launch_bounds__(kWideThreads, 2)
wide_upsweep_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ counts,
                    uint32_t nblocks, bool vec, const unsigned long long* __restrict__ n_dev,
                    const unsigned long long* __restrict__ base_dev) {
    constexpr int kBins = 1 << kBits;
    __shared__ uint32_t hist[kBins];
    if (base_dev) {
        keys += *base_dev;
        vec = vec && ((uintptr_t)keys & 15) == 0;
    }
    for (int d = threadIdx.x; d < kBins; d += kWideThreads) hist[d] = 0;
    __syncthreads();
    int64_t lo, hi;
    wide_range(n, n_dev, nblocks, lo, hi);
    hist_runs<kWideThreads, (uint32_t)(kBins - 1)>(keys, lo, hi, shift, vec, hist);
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += kWideThreads) counts[(int64_t)d * nblocks + blockIdx.x] = hist[d];
}

template <int kBits>
__global__ void __launch_bounds__(kWideThreads, 2)
wide_downsweep_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
                      uint32_t* __restrict__ vout, int64_t n, int shift, const uint32_t* __restrict__ offsets,
                      uint32_t nblocks, const unsigned long long* __restrict__ n_dev,
                      const unsigned long long* __restrict__ base_dev) {
    constexpr int kBins = 1 << kBits;
    constexpr uint32_t kMask = (uint32_t)kBins - 1u;
    if (base_dev) {
        const unsigned long long b = *base_dev;
        kin += b; vin += b; kout += b; vout += b;
    }
    constexpr int kPer = kBins / kWideThreads > 0 ? kBins / kWideThreads : 1;   // digits per thread in the scan
    extern __shared__ __align__(16) unsigned char wide_smem_raw[];
    WideSmem<kBits>& sm = *reinterpret_cast<WideSmem<kBits>*>(wide_smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* wh = reinterpret_cast<uint32_t*>(&sm.whist[0][0]);
    for (int i = threadIdx.x; i < kWideWarps * kBins / 2; i += kWideThreads) wh[i] = 0u;
    for (int d = threadIdx.x; d < kBins; d += kWideThreads) sm.goff[d] = offsets[(int64_t)d * nblocks + blockIdx.x];
    int64_t lo, hi;
    wide_range(n, n_dev, nblocks, lo, hi);
    // warp w holds tile items [w*512, (w+1)*512) in 16 rounds of 32 lanes: (round, lane)
    // order is input order.  The values are read only when the keys are placed (registers),
    // and the next tile's keys are read while this tile is written out.
    uint32_t key[kWideItems];
    auto load_keys = [&](int64_t base, int count) {
#pragma unroll
        for (int r = 0; r < kWideItems; ++r) {
            const int li = warp * (kWideItems * 32) + r * 32 + lane;
            key[r] = li < count ? kin[base + li] : 0u;
        }
    };
    if (lo < hi) load_keys(lo, hi - lo < kWideTile ? (int)(hi - lo) : kWideTile);
    __syncthreads();
    for (int64_t base = lo; base < hi; base += kWideTile) {   // tiles in order: stable
        const int count = hi - base < kWideTile ? (int)(hi - base) : kWideTile;
        uint32_t rank2[kWideItems / 2];   // ranks within the warp, two 16-bit halves per word
#pragma unroll
        for (int r = 0; r < kWideItems; ++r) {
            const int li = warp * (kWideItems * 32) + r * 32 + lane;
            const uint32_t dig = li < count ? (key[r] >> shift) & kMask : (uint32_t)kBins;
            const unsigned peers = __match_any_sync(0xffffffffu, dig);
            const unsigned lower = peers & ((1u << lane) - 1u);
            const uint32_t prior = dig < (uint32_t)kBins ? (uint32_t)sm.whist[warp][dig] : 0u;
            const uint32_t rk = prior + (uint32_t)__popc(lower);
            if (r & 1) rank2[r >> 1] |= rk << 16;
            else rank2[r >> 1] = rk;
            __syncwarp();
            if (dig < (uint32_t)kBins && lower == 0u)
                sm.whist[warp][dig] = (uint16_t)(prior + (uint32_t)__popc(peers));
            __syncwarp();
        }
        __syncthreads();
        // the tile's digit totals, their exclusive scan (thread t owns digits
        // [t kPer, t kPer + kPer)), then each (warp, digit)'s first slot in the tile
        for (int d = threadIdx.x; d < kBins; d += kWideThreads) {
            uint32_t t = 0;
#pragma unroll
            for (int w = 0; w < kWideWarps; ++w) t += sm.whist[w][d];
            sm.dtot[d] = t;
        }
        __syncthreads();
        {
            const int d0 = threadIdx.x * kPer;
            uint32_t loc = 0, v[kPer];
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                v[j] = d0 < kBins ? sm.dtot[d0 + j] : 0u;
                loc += v[j];
            }
            uint32_t incl = loc;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) sm.wsum[warp] = incl;
            __syncthreads();
            uint32_t run = incl - loc;
            for (int w = 0; w < warp; ++w) run += sm.wsum[w];
            if (d0 < kBins) {
#pragma unroll
                for (int j = 0; j < kPer; ++j) {
                    const int d = d0 + j;
                    uint32_t slot = run;
#pragma unroll
                    for (int w = 0; w < kWideWarps; ++w) {
                        const uint32_t c = sm.whist[w][d];
                        sm.whist[w][d] = (uint16_t)slot;
                        slot += c;
                    }
                    sm.gbase[d] = sm.goff[d] - run;
                    sm.goff[d] += v[j];
                    run += v[j];
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kWideItems; ++r) {
            const int li = warp * (kWideItems * 32) + r * 32 + lane;
            if (li < count) {
                const uint32_t dig = (key[r] >> shift) & kMask;
                const uint32_t rk = (r & 1) ? rank2[r >> 1] >> 16 : rank2[r >> 1] & 0xFFFFu;
                const uint32_t pos = (uint32_t)sm.whist[warp][dig] + rk;
                sm.skeys[pos] = key[r];
                sm.svals[pos] = vin[base + li];
            }
        }
        __syncthreads();
        const int64_t next = base + kWideTile;
        if (next < hi) load_keys(next, hi - next < kWideTile ? (int)(hi - next) : kWideTile);
        for (int i = threadIdx.x; i < count; i += kWideThreads) {
            const uint32_t k = sm.skeys[i];
            const uint32_t o = sm.gbase[(k >> shift) & kMask] + (uint32_t)i;
            kout[o] = k;
            vout[o] = sm.svals[i];
        }
        for (int i = threadIdx.x; i < kWideWarps * kBins / 2; i += kWideThreads) wh[i] = 0u;
        __syncthreads();   // the next tile ranks into whist and rewrites gbase, skeys and svals
    }
}

// n_dev (nullable): the key count lives in device memory and n is the capacity; the grid
// is then kWideChunks blocks (stream-capturable).  base_dev (nullable, with n_dev): the
// keys start at that element of the arrays (a device value).
template <int kBits>
int wide_pass(const uint32_t* ka, const uint32_t* va, uint32_t* kb, uint32_t* vb, int64_t n, int shift,
              uint32_t* counts, void* stemp, size_t sbytes, cudaStream_t s,
              const unsigned long long* n_dev = nullptr, const unsigned long long* base_dev = nullptr) {
    constexpr int kBins = 1 << kBits;
    const int64_t nb = n_dev ? kWideChunks : (n + kWideBlockItems - 1) / kWideBlockItems;
    const int64_t nc = nb * kBins;
    const size_t smem = sizeof(WideSmem<kBits>);
    // the attribute belongs to the function on the current device; it is set on every call
    // outside a stream capture (a driver call per pass), and by sort_prepare before one
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    RGS_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
    if (cap == cudaStreamCaptureStatusNone)
        RGS_CUDA_TRY(cudaFuncSetAttribute(wide_downsweep_kernel<kBits>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
    wide_upsweep_kernel<kBits><<<(unsigned)nb, kWideThreads, 0, s>>>(ka, n, shift, counts, (uint32_t)nb,
                                                                      ((uintptr_t)ka & 15) == 0, n_dev, base_dev);
    RGS_CUDA_LAUNCH_CHECK();
    int rc = exclusive_scan_u32(counts, counts, nc, 0, nullptr, stemp, sbytes, s);
    if (rc != RGS_OK) return rc;
    wide_downsweep_kernel<kBits><<<(unsigned)nb, kWideThreads, smem, s>>>(ka, va, kb, vb, n, shift, counts,
                                                                           (uint32_t)nb, n_dev, base_dev);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

// ------------------------------------------------------------------ device-counted passes
// Variants whose element count is read from device memory (a counter written by an
// earlier kernel on the stream), so that the launches need no host round trip and can
// be captured in a CUDA graph.  The grid is fixed: block c owns the c-th of kChunks
// contiguous chunks (whole tiles) of [0, n) and walks its tiles in order, so scans and
// sorts stay stable.
// A fixed chunk count (it sizes the count tables and the graph's launches): four resident
// blocks on each SM of a GB300 (152 SMs); on a device with other SM counts only the
// balance of the chunks changes, not the result.
constexpr int kChunks = 608;

__device__ __forceinline__ void chunk_range(int64_t n, int64_t tile, int64_t& lo, int64_t& hi) {
    const int64_t tiles = (n + tile - 1) / tile;
    const int64_t per = (tiles + kChunks - 1) / kChunks;
    lo = min(n, (int64_t)blockIdx.x * per * tile);
    hi = min(n, lo + per * tile);
}

__device__ __forceinline__ int64_t device_count(const unsigned long long* n_dev, int64_t cap) {
    const unsigned long long v = *n_dev;
    return v < (unsigned long long)cap ? (int64_t)v : cap;
}

__global__ void __launch_bounds__(kScanThreads)
dscan_reduce_kernel(const uint32_t* __restrict__ in, const unsigned long long* __restrict__ n_dev, int64_t cap,
                    int mode, const uint32_t* __restrict__ gather, uint32_t* __restrict__ sums) {
    int64_t lo, hi;
    chunk_range(device_count(n_dev, cap), kScanTile, lo, hi);
    uint32_t acc = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kScanThreads) acc += load_item(in, gather, i, mode);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ uint32_t ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kScanThreads)
dscan_tile_kernel(const uint32_t* in, uint32_t* out, const unsigned long long* __restrict__ n_dev, int64_t cap,
                  int mode, const uint32_t* __restrict__ gather, const uint32_t* __restrict__ chunk_offsets) {
    int64_t lo, hi;
    const int64_t n = device_count(n_dev, cap);
    chunk_range(n, kScanTile, lo, hi);
    uint32_t off = chunk_offsets[blockIdx.x];
    for (int64_t base = lo; base < hi; base += kScanTile) off += scan_tile_body(in, out, hi, mode, gather, base, off);
}

__global__ void __launch_bounds__(kSortThreads, 4)
dradix_upsweep_kernel(const uint32_t* __restrict__ keys, const unsigned long long* __restrict__ n_dev, int64_t cap,
                      int shift, uint32_t* __restrict__ counts, const unsigned long long* __restrict__ base_dev) {
    __shared__ uint32_t hist[kRadix];
    if (base_dev) keys += *base_dev;
    hist[threadIdx.x] = 0;
    __syncthreads();
    int64_t lo, hi;
    chunk_range(device_count(n_dev, cap), kSortTile, lo, hi);
    hist_runs(keys, lo, hi, shift, ((uintptr_t)keys & 15) == 0, hist);
    __syncthreads();
    counts[(int64_t)threadIdx.x * kChunks + blockIdx.x] = hist[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads, 4)
dradix_downsweep_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
                        uint32_t* __restrict__ vout, const unsigned long long* __restrict__ n_dev, int64_t cap,
                        int shift, const uint32_t* __restrict__ offsets,
                        const unsigned long long* __restrict__ base_dev) {
    __shared__ uint32_t goff[kRadix];
    if (base_dev) {
        const unsigned long long b = *base_dev;
        kin += b; vin += b; kout += b; vout += b;
    }
    goff[threadIdx.x] = offsets[(int64_t)threadIdx.x * kChunks + blockIdx.x];
    int64_t lo, hi;
    chunk_range(device_count(n_dev, cap), kSortTile, lo, hi);
    for (int64_t base = lo; base < hi; base += kSortTile) {
        const int64_t rem = hi - base;
        radix_tile_body(kin, vin, kout, vout, base, rem < kSortTile ? (int)rem : kSortTile, shift, goff);
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

size_t scan_temp_bytes(int64_t n) {
    size_t total = 0;
    int64_t m = cdiv(n, kScanTile);
    while (m > 1) {
        total += align256((size_t)m * 4);
        m = cdiv(m, kScanTile);
    }
    return total + 256;
}

int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, int load, const uint32_t* gather, void* temp,
                       size_t temp_bytes, cudaStream_t s) {
    if (n <= 0) return RGS_OK;
    int64_t nb = cdiv(n, kScanTile);
    if (nb == 1) {
        scan_tile_kernel<<<1, kScanThreads, 0, s>>>(in, out, n, load, gather, nullptr);
        RGS_CUDA_LAUNCH_CHECK();
        return RGS_OK;
    }
    size_t need = align256((size_t)nb * 4);
    if (need > temp_bytes) {
        set_error("scan: temporary buffer too small (%zu < %zu)", temp_bytes, need);
        return RGS_EOVERFLOW;
    }
    uint32_t* sums = (uint32_t*)temp;
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, load, gather, sums);
    RGS_CUDA_LAUNCH_CHECK();
    int rc = exclusive_scan_u32(sums, sums, nb, 0, nullptr, (char*)temp + need, temp_bytes - need, s);
    if (rc != RGS_OK) return rc;
    scan_tile_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, load, gather, sums);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

size_t radix_temp_bytes(int64_t n) {
    const int64_t nc8 = cdiv(n > 0 ? n : 1, kBlockItems) * kRadix;
    const int64_t ncw = cdiv(n > 0 ? n : 1, kWideBlockItems) * ((int64_t)1 << kWideMaxBits);
    const int64_t nc = nc8 > ncw ? nc8 : ncw;
    return align256((size_t)nc * 4) + scan_temp_bytes(nc);
}

int radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, int64_t n, int end_bit,
                     void* temp, size_t temp_bytes, cudaStream_t s, bool* in_alt) {
    *in_alt = false;
    if (n <= 1 || end_bit <= 0) return RGS_OK;
    if (n > 0xFFFFFFFFll) {
        set_error("radix sort: %lld elements exceed the 32-bit index range", (long long)n);
        return RGS_EOVERFLOW;
    }
    int64_t nb = cdiv(n, kBlockItems);
    int64_t nc = nb * kRadix;
    const int64_t ncw = cdiv(n, kWideBlockItems) * ((int64_t)1 << kWideMaxBits);
    size_t cbytes = align256((size_t)(nc > ncw ? nc : ncw) * 4);
    if (temp_bytes < cbytes + scan_temp_bytes(nc > ncw ? nc : ncw)) {
        set_error("radix sort: temporary buffer too small");
        return RGS_EOVERFLOW;
    }
    uint32_t* counts = (uint32_t*)temp;
    void* stemp = (char*)temp + cbytes;
    size_t sbytes = temp_bytes - cbytes;
    uint32_t *ka = keys, *va = vals, *kb = keys_alt, *vb = vals_alt;
    if (end_bit > 2 * kRadixBits && end_bit <= 2 * kWideMaxBits) {
        // two wide passes: the low ceil(end_bit / 2) bits, then the rest
        const int b0 = (end_bit + 1) / 2;
        int shift = 0;
        for (int pass = 0; pass < 2; ++pass) {
            const int bits = pass == 0 ? b0 : end_bit - b0;
            int rc = bits == 10   ? wide_pass<10>(ka, va, kb, vb, n, shift, counts, stemp, sbytes, s)
                     : bits == 9  ? wide_pass<9>(ka, va, kb, vb, n, shift, counts, stemp, sbytes, s)
                                  : wide_pass<8>(ka, va, kb, vb, n, shift, counts, stemp, sbytes, s);
            if (rc != RGS_OK) return rc;
            shift += bits;
            uint32_t* t;
            t = ka; ka = kb; kb = t;
            t = va; va = vb; vb = t;
            *in_alt = !*in_alt;
        }
        return RGS_OK;
    }
    for (int shift = 0; shift < end_bit; shift += kRadixBits) {
        radix_upsweep_kernel<<<(unsigned)nb, kSortThreads, 0, s>>>(ka, n, shift, counts, (uint32_t)nb,
                                                                   ((uintptr_t)ka & 15) == 0);
        RGS_CUDA_LAUNCH_CHECK();
        int rc = exclusive_scan_u32(counts, counts, nc, 0, nullptr, stemp, sbytes, s);
        if (rc != RGS_OK) return rc;
        radix_downsweep_kernel<<<(unsigned)nb, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift, counts, (uint32_t)nb);
        RGS_CUDA_LAUNCH_CHECK();
        uint32_t* t;
        t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
        *in_alt = !*in_alt;
    }
    return RGS_OK;
}

size_t scan_dev_temp_bytes() { return align256((size_t)kChunks * 4) + 256; }

int exclusive_scan_dev(const uint32_t* in, uint32_t* out, const unsigned long long* n_dev, int64_t cap, int load,
                       const uint32_t* gather, void* temp, size_t temp_bytes, cudaStream_t s) {
    static_assert(kChunks <= kScanTile, "chunk sums are scanned by one block");
    if (cap <= 0) return RGS_OK;
    if (temp_bytes < scan_dev_temp_bytes()) {
        set_error("scan: temporary buffer too small");
        return RGS_EOVERFLOW;
    }
    uint32_t* sums = (uint32_t*)temp;
    dscan_reduce_kernel<<<kChunks, kScanThreads, 0, s>>>(in, n_dev, cap, load, gather, sums);
    RGS_CUDA_LAUNCH_CHECK();
    scan_tile_kernel<<<1, kScanThreads, 0, s>>>(sums, sums, kChunks, 0, nullptr, nullptr);
    RGS_CUDA_LAUNCH_CHECK();
    dscan_tile_kernel<<<kChunks, kScanThreads, 0, s>>>(in, out, n_dev, cap, load, gather, sums);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int sort_prepare() {
    RGS_CUDA_TRY(cudaFuncSetAttribute(wide_downsweep_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(WideSmem<8>)));
    RGS_CUDA_TRY(cudaFuncSetAttribute(wide_downsweep_kernel<9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(WideSmem<9>)));
    RGS_CUDA_TRY(cudaFuncSetAttribute(wide_downsweep_kernel<10>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(WideSmem<10>)));
    return RGS_OK;
}

size_t radix_dev_temp_bytes() {
    const int64_t nc8 = (int64_t)kRadix * kChunks, ncw = ((int64_t)1 << kWideMaxBits) * kWideChunks;
    const int64_t nc = nc8 > ncw ? nc8 : ncw;
    return align256((size_t)nc * 4) + scan_temp_bytes(nc);
}

int radix_sort_pairs_dev(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                         const unsigned long long* n_dev, int64_t cap, int end_bit, void* temp, size_t temp_bytes,
                         cudaStream_t s, bool* in_alt, const unsigned long long* base_dev) {
    static_assert(kRadix == kSortThreads, "one digit per thread");
    *in_alt = false;
    if (cap <= 1 || end_bit <= 0) return RGS_OK;
    if (cap > 0xFFFFFFFFll) {
        set_error("radix sort: capacity %lld exceeds the 32-bit index range", (long long)cap);
        return RGS_EOVERFLOW;
    }
    const int64_t nc = (int64_t)kRadix * kChunks, ncw = ((int64_t)1 << kWideMaxBits) * kWideChunks;
    const size_t cbytes = align256((size_t)(nc > ncw ? nc : ncw) * 4);
    if (temp_bytes < radix_dev_temp_bytes()) {
        set_error("radix sort: temporary buffer too small");
        return RGS_EOVERFLOW;
    }
    uint32_t* counts = (uint32_t*)temp;
    void* stemp = (char*)temp + cbytes;
    const size_t sbytes = temp_bytes - cbytes;
    uint32_t *ka = keys, *va = vals, *kb = keys_alt, *vb = vals_alt;
    if (end_bit > 2 * kRadixBits && end_bit <= 2 * kWideMaxBits) {
        // two wide passes, as radix_sort_pairs
        const int b0 = (end_bit + 1) / 2;
        int shift = 0;
        for (int pass = 0; pass < 2; ++pass) {
            const int bits = pass == 0 ? b0 : end_bit - b0;
            int rc = bits == 10   ? wide_pass<10>(ka, va, kb, vb, cap, shift, counts, stemp, sbytes, s, n_dev, base_dev)
                     : bits == 9  ? wide_pass<9>(ka, va, kb, vb, cap, shift, counts, stemp, sbytes, s, n_dev, base_dev)
                                  : wide_pass<8>(ka, va, kb, vb, cap, shift, counts, stemp, sbytes, s, n_dev, base_dev);
            if (rc != RGS_OK) return rc;
            shift += bits;
            uint32_t* t;
            t = ka; ka = kb; kb = t;
            t = va; va = vb; vb = t;
            *in_alt = !*in_alt;
        }
        return RGS_OK;
    }
    for (int shift = 0; shift < end_bit; shift += kRadixBits) {
        dradix_upsweep_kernel<<<kChunks, kSortThreads, 0, s>>>(ka, n_dev, cap, shift, counts, base_dev);
        RGS_CUDA_LAUNCH_CHECK();
        int rc = exclusive_scan_u32(counts, counts, nc, 0, nullptr, stemp, sbytes, s);
        if (rc != RGS_OK) return rc;
        dradix_downsweep_kernel<<<kChunks, kSortThreads, 0, s>>>(ka, va, kb, vb, n_dev, cap, shift, counts, base_dev);
        RGS_CUDA_LAUNCH_CHECK();
        uint32_t* t;
        t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
        *in_alt = !*in_alt;
    }
    return RGS_OK;
}

}  // namespace rgs
