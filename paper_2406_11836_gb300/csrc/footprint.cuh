// Screen-space footprint of a projected splat: the pixels whose centre can pass the
// truncation tests of a (pixel, splat) pair, i.e. the ellipse d^2 <= d2max of the 2D
// Gaussian (d2max = min(trunc^2, 2 ln(alpha / alpha_min)): beyond it sigma < alpha_min)
// intersected with the ball test (dx/fx)^2 + (dy/fy)^2 <= (D/z)^2.  Used, with identical
// arithmetic on identical inputs, to count a splat's tile instances, to emit them, and to
// mark which warp blocks of a tile a staged record can touch; the margins make it a
// superset of what the fp32 per-pair tests accept.
#pragma once

#include "rgs_internal.cuh"

namespace rgs {

struct Footprint {
    float cx, cy;            // centre (pixels; hi part of the projected centre)
    float qa, qb, qc, det;   // conic Q = [[qa, qb], [qb, qc]] = L^T L, det = det(Q)
    float r2;                // d2max with margin
    float ex, ey;            // ellipse half-extents
    float bx, by;            // ball half-extents (pixels)
    float rho2;              // (D/z)^2 with margin
    float ystar;             // y offset of the ellipse's rightmost point
    float zr;                // foot reading: half-width of the foot's depth interval (0: depth plane)
    bool empty;
};

// Foot reading: a foot that passes the ball test lies within D of the centre, so its
// camera depth lies within D of z.  D = z sqrt(rho2) from the ball radius rho2 = (D/z)^2,
// widened by 0.1%; the count and the emission evaluate this on the same stored values.
__device__ __forceinline__ float foot_depth_radius(float z, float rho2_ball) {
    return __fmul_rn(__fmul_rn(z, __fsqrt_rn(rho2_ball)), 1.001f);
}

__device__ __forceinline__ Footprint make_footprint(float mxh, float myh, float l11, float l12, float l22, float alpha,
                                                    float rho2_signed, const ViewParams& vp) {
    Footprint f;
    f.cx = mxh;
    f.cy = myh;
    f.qa = l11 * l11;
    f.qb = l11 * l12;
    f.qc = fmaf(l12, l12, l22 * l22);
    const float sd = l11 * l22;
    f.det = sd * sd;
    float d2max = fminf(vp.trunc_mult * vp.trunc_mult, 2.f * __logf(alpha / vp.alpha_min));
    f.empty = !(d2max >= 0.f);
    f.r2 = fmaxf(d2max, 0.f) * 1.002f + 2e-3f;
    // covariance = Q^{-1}: xx = qc/det, yy = qa/det, xy = -qb/det
    const float idet = 1.f / f.det;
    const float sxx = f.qc * idet, syy = f.qa * idet, sxy = -f.qb * idet;
    f.ex = sqrtf(f.r2 * sxx);
    f.ey = sqrtf(f.r2 * syy);
    f.ystar = sqrtf(f.r2) * sxy * rsqrtf(sxx);
    f.rho2 = fabsf(rho2_signed) * 1.002f;
    const float rb = sqrtf(f.rho2);
    f.bx = vp.fx * rb;
    f.by = vp.fy * rb;
    f.zr = 0.f;
    return f;
}

// Horizontal extent [x0, x1] (offsets from the centre) of the footprint over the band of
// pixel-centre offsets y in [ylo, yhi].  Returns false if the band misses it.
__device__ __forceinline__ bool footprint_span(const Footprint& f, const ViewParams& vp, float ylo, float yhi,
                                               float& x0, float& x1) {
    const float yl = fmaxf(ylo, fmaxf(-f.ey, -f.by)), yh = fminf(yhi, fminf(f.ey, f.by));
    if (!(yl <= yh)) return false;
    // ellipse: x(y) = (-qb y +- sqrt(qa r2 - det y^2)) / qa; the right branch is concave and
    // peaks at ystar, the left branch is convex with its minimum at -ystar
    const float yr = fminf(fmaxf(f.ystar, yl), yh);
    const float yq = fminf(fmaxf(-f.ystar, yl), yh);
    const float iqa = 1.f / f.qa;
    const float xr = fmaf(-f.qb, yr, sqrtf(fmaxf(fmaf(-f.det, yr * yr, f.qa * f.r2), 0.f))) * iqa;
    const float xl = fmaf(-f.qb, yq, -sqrtf(fmaxf(fmaf(-f.det, yq * yq, f.qa * f.r2), 0.f))) * iqa;
    // ball: widest where |y| is smallest
    const float y0 = fminf(fmaxf(0.f, yl), yh) * vp.ify;
    const float xb = vp.fx * sqrtf(fmaxf(f.rho2 - y0 * y0, 0.f));
    x0 = fmaxf(xl, -xb) - 0.02f;
    x1 = fminf(xr, xb) + 0.02f;
    return x0 <= x1;
}

// Rows of tiles the footprint can touch.
__device__ __forceinline__ void footprint_tile_rows(const Footprint& f, const ViewParams& vp, int& ty0, int& ty1) {
    const float h = fminf(f.ey, f.by) + 0.02f;
    ty0 = (int)fmaxf(floorf((f.cy - h - 0.5f) * (1.f / kTile)), 0.f);
    ty1 = (int)fminf(floorf((f.cy + h - 0.5f) * (1.f / kTile)), (float)(vp.tiles_y - 1));
}

// Tile columns [c0, c1] the footprint touches in tile row ty (c0 > c1: none).
__device__ __forceinline__ void footprint_row_tiles(const Footprint& f, const ViewParams& vp, int ty, int& c0, int& c1) {
    const float ylo = (float)(ty * kTile) + 0.5f - f.cy, yhi = (float)(ty * kTile) + (kTile - 0.5f) - f.cy;
    float x0, x1;
    if (!footprint_span(f, vp, ylo, yhi, x0, x1)) {
        c0 = 1;
        c1 = 0;
        return;
    }
    // pixel columns px with centre px + 0.5 in [cx + x0, cx + x1]
    c0 = (int)fmaxf(floorf(ceilf(f.cx + x0 - 0.5f) * (1.f / kTile)), 0.f);
    c1 = (int)fminf(floorf(floorf(f.cx + x1 - 0.5f) * (1.f / kTile)), (float)(vp.tiles_x - 1));
}

// ------------------------------------------------------------------ plane test (Eq. 6)
// For a splat at camera depth z, the ray point x_i = o + z d_p of the pixel with centre
// (X, Y) has x_i[a] - s = A X + B Y + C along a node's axis.  The blend decides "x_i on
// the right of the node" as A X + B Y + C >= 0 with these coefficients, computed by this one
// function for every leaf that tests the node, so the leaves' decisions are complementary
// and every (pixel, splat) pair lands in exactly one subset.
__device__ __forceinline__ float4 plane_coeffs(const ViewParams& vp, int a, float s, float z) {
    const float Ra = vp.R[a], Rb = vp.R[3 + a], Rc = vp.R[6 + a];
    const float oa = a == 0 ? vp.o[0] : (a == 1 ? vp.o[1] : vp.o[2]);
    const float gam = Rc - Ra * vp.cx * vp.ifx - Rb * vp.cy * vp.ify;
    return make_float4(z * Ra * vp.ifx, z * Rb * vp.ify, fmaf(z, gam, oa - s), 0.f);
}

// ------------------------------------------------------------------ subset clipping (Eq. 6)
// The L plane constraints of one KD leaf.
struct LeafPath {
    float split[kMaxRenderDepth];
    int axis_right[kMaxRenderDepth];   // axis | (right << 2)
};

__device__ __forceinline__ void leaf_path(const TreeParams& tp, int k, LeafPath& lp) {
    int node = 0;
#pragma unroll
    for (int d = 0; d < kMaxRenderDepth; ++d) {
        if (d >= tp.L) break;
        const int right = (k >> (tp.L - 1 - d)) & 1;
        lp.split[d] = tp.split[node];
        lp.axis_right[d] = tp.axis[node] | (right << 2);
        node = 2 * node + 1 + right;
    }
}

// For a splat at camera depth z, the point x_i = o + z d_p of pixel-centre (X, Y) has
// coordinate x_i[a] = A X + B Y + C + s along the split's axis (d_p is affine in X, Y), so
// each plane of the leaf is a half-plane of the image: sign * (A X + B Y + C) >= 0 with
// sign +1 on the right branch and -1 on the left.  `m` is a margin in world units, far
// above the fp32 error of the per-pixel test, so clipping never drops a pixel the test
// would accept.
struct SubsetClip {
    int n;
    float A[kMaxRenderDepth], B[kMaxRenderDepth], C[kMaxRenderDepth], m[kMaxRenderDepth];
};

__device__ __forceinline__ void make_clip(const ViewParams& vp, const LeafPath& lp, int L, float z, SubsetClip& c) {
    c.n = L;
#pragma unroll
    for (int d = 0; d < kMaxRenderDepth; ++d) {
        if (d >= L) break;
        const int ar = lp.axis_right[d];
        const int a = ar & 3;
        const float sg = (ar >> 2) ? 1.f : -1.f;
        const float Ra = vp.R[a], Rb = vp.R[3 + a], Rc = vp.R[6 + a];
        const float oa = a == 0 ? vp.o[0] : (a == 1 ? vp.o[1] : vp.o[2]);
        const float s = lp.split[d];
        const float gam = Rc - Ra * vp.cx * vp.ifx - Rb * vp.cy * vp.ify;
        c.A[d] = sg * z * Ra * vp.ifx;
        c.B[d] = sg * z * Rb * vp.ify;
        c.C[d] = sg * (fmaf(z, gam, oa) - s);
        c.m[d] = 1e-5f * (fabsf(oa) + fabsf(s) + 4.f * z) + 1e-6f;
    }
}

// The same half-planes from the view's plane templates: for subset k and level d of its
// leaf path, tab (tA, tB, tG, tC) and margin m0 with the branch sign folded in, so that
// the plane at depth z is (z tA) X + (z tB) Y + (z tG + tC) >= 0 with margin m0 + 4e-5 z.
// No tree walk and no per-axis selection per item: the count and the emission call this
// on the same inputs, so they agree.
__device__ __forceinline__ void make_clip_tab(const ViewParams& vp, int k, int L, float z, SubsetClip& c) {
    c.n = L;
    const float4* t = vp.clip_plane() + k * L;
    const float* tm = vp.clip_margin() + k * L;
#pragma unroll
    for (int d = 0; d < kMaxRenderDepth; ++d) {
        if (d >= L) break;
        const float4 q = __ldg(t + d);
        c.A[d] = z * q.x;
        c.B[d] = z * q.y;
        c.C[d] = fmaf(z, q.z, q.w);
        c.m[d] = fmaf(4e-5f, z, __ldg(tm + d));
    }
}

// Narrow [xlo, xhi] (absolute pixel-centre X) to the X where, for some Y in [ylo, yhi],
// every half-plane holds within its margin.  Returns false if nothing is left.
__device__ __forceinline__ bool clip_span(const SubsetClip& c, float ylo, float yhi, float& xlo, float& xhi) {
#pragma unroll
    for (int d = 0; d < kMaxRenderDepth; ++d) {
        if (d >= c.n) break;
        const float by = fmaxf(c.B[d] * ylo, c.B[d] * yhi);
        const float rhs = -c.m[d] - c.C[d] - by;       // need A X >= rhs
        // approximate division: its error (a few ulp of X) is far below the margin m / |A|
        if (c.A[d] > 0.f) xlo = fmaxf(xlo, __fdividef(rhs, c.A[d]));
        else if (c.A[d] < 0.f) xhi = fminf(xhi, __fdividef(rhs, c.A[d]));
        else if (rhs > 0.f) return false;
    }
    return xlo <= xhi;
}

// The same narrowing for a point anywhere on the pixel ray between depths za and zb
// (0 < za < zb): the point's coordinate along a split axis is affine in its depth, so a
// half-plane holds somewhere in between iff it holds at za or at zb; per plane the looser
// of the two half-lines (both point the same way, the slope having the sign of the depth)
// is kept.  Reads the view's plane templates for subset k directly.
__device__ __forceinline__ bool clip_span_depths(const ViewParams& vp, int k, int L, float za, float zb, float ylo,
                                                 float yhi, float& xlo, float& xhi) {
    const float4* t = vp.clip_plane() + k * L;
    const float* tm = vp.clip_margin() + k * L;
    const float inf = __int_as_float(0x7f800000);
#pragma unroll
    for (int d = 0; d < kMaxRenderDepth; ++d) {
        if (d >= L) break;
        const float4 q = __ldg(t + d);
        const float m0 = __ldg(tm + d);
        float lo = inf, hi = -inf;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float z = e ? zb : za;
            const float A = z * q.x, B = z * q.y, C = fmaf(z, q.z, q.w), m = fmaf(4e-5f, z, m0);
            const float rhs = -m - C - fmaxf(B * ylo, B * yhi);   // need A X >= rhs
            if (A > 0.f) {
                lo = fminf(lo, __fdividef(rhs, A));
                hi = inf;
            } else if (A < 0.f) {
                hi = fmaxf(hi, __fdividef(rhs, A));
                lo = -inf;
            } else if (rhs <= 0.f) {
                lo = -inf;
                hi = inf;
            }
        }
        xlo = fmaxf(xlo, lo);
        xhi = fminf(xhi, hi);
    }
    return xlo <= xhi;
}

// Foot reading: the camera depth of the foot for pixel centres in [X0, X1] x [Y0, Y1] is
// z (1 + r_x u_x + r_y u_y) / (1 + r_x^2 + r_y^2), u the projected centre in normalised
// units; bounded by the extremes of the linear numerator and of the quadratic denominator
// over the rectangle, intersected with [z - zr, z + zr] and widened by 1e-4.  Returns
// false when the range reaches the camera (then nothing is clipped).
__device__ __forceinline__ bool foot_depth_range(const Footprint& f, const ViewParams& vp, float z, float X0, float X1,
                                                 float Y0, float Y1, float& za, float& zb) {
    const float ux = (f.cx - vp.cx) * vp.ifx, uy = (f.cy - vp.cy) * vp.ify;
    const float rx0 = (X0 - vp.cx) * vp.ifx, rx1 = (X1 - vp.cx) * vp.ifx;
    const float ry0 = (Y0 - vp.cy) * vp.ify, ry1 = (Y1 - vp.cy) * vp.ify;
    const float nlo = 1.f + fminf(rx0 * ux, rx1 * ux) + fminf(ry0 * uy, ry1 * uy);
    const float nhi = 1.f + fmaxf(rx0 * ux, rx1 * ux) + fmaxf(ry0 * uy, ry1 * uy);
    const float qhi = 1.f + fmaxf(rx0 * rx0, rx1 * rx1) + fmaxf(ry0 * ry0, ry1 * ry1);
    const float qlo = 1.f + (rx0 * rx1 <= 0.f ? 0.f : fminf(rx0 * rx0, rx1 * rx1)) +
                      (ry0 * ry1 <= 0.f ? 0.f : fminf(ry0 * ry0, ry1 * ry1));
    za = fmaxf(z - f.zr, z * nlo / qhi) * (1.f - 1e-4f);
    zb = fminf(z + f.zr, z * nhi / qlo) * (1.f + 1e-4f);
    return nlo > 0.f && za > 0.f && za <= zb;
}

// Tile columns [c0, c1] of tile row ty touched by the footprint restricted to subset clip
// `c` (c == nullptr: no restriction).
__device__ __forceinline__ void footprint_row_tiles_clipped(const Footprint& f, const ViewParams& vp, int ty,
                                                            const SubsetClip* c, int& c0, int& c1) {
    const float Ylo = (float)(ty * kTile) + 0.5f, Yhi = (float)(ty * kTile) + (kTile - 0.5f);
    float x0, x1;
    c0 = 1;
    c1 = 0;
    if (!footprint_span(f, vp, Ylo - f.cy, Yhi - f.cy, x0, x1)) return;
    float X0 = f.cx + x0, X1 = f.cx + x1;
    if (c && !clip_span(*c, Ylo, Yhi, X0, X1)) return;
    c0 = (int)fmaxf(floorf(ceilf(X0 - 0.5f) * (1.f / kTile)), 0.f);
    c1 = (int)fminf(floorf(floorf(X1 - 0.5f) * (1.f / kTile)), (float)(vp.tiles_x - 1));
}

// Item `it` of a splat (subset index it / rows, tile row ty0 + it % rows): its tile row,
// its subset k and the tile columns [c0, c1] the footprint touches there, clipped to the
// subset when the splat is held by several (Eq. 6).  The count in the projection and the
// emission call this same function on the same record values, so they always agree.
// Item `it` of a splat: (subset k, tile row ty), subsets in mask order, rows inner.
__device__ __forceinline__ void item_locate(unsigned long long mask, int ty0, int rows, int it, int& ty, int& k) {
    const int si = it / rows;
    ty = ty0 + (it - si * rows);
    unsigned long long mm = mask;
    for (int q = 0; q < si; ++q) mm &= mm - 1;
    k = __ffsll((long long)mm) - 1;
}

// Tile columns [c0, c1] of the item's row for subset k (clipped to the subset when the
// splat straddles).  kMulti = 0: the splat is known to lie in one subset (no clipping code
// is compiled in); 1: it is known to straddle; -1: decided at run time.
template <int kMulti = -1>
__device__ __forceinline__ void item_cols(const Footprint& f, const ViewParams& vp, const TreeParams& tp, int k,
                                          int nsub, float z, int ty, int& c0, int& c1) {
    if (kMulti == 1 || (kMulti < 0 && nsub > 1)) {
        if (f.zr > 0.f) {
            // foot reading: clip with the foot's depth range over the row's span, twice (the
            // second time over the narrowed span); nothing is clipped where that range
            // reaches the camera
            footprint_row_tiles_clipped(f, vp, ty, nullptr, c0, c1);
            const float Ylo = (float)(ty * kTile) + 0.5f, Yhi = (float)(ty * kTile) + (kTile - 0.5f);
            for (int pass = 0; pass < 2 && c0 <= c1; ++pass) {
                float X0 = (float)(c0 * kTile) + 0.5f, X1 = (float)(c1 * kTile) + (kTile - 0.5f);
                float za, zb;
                if (!foot_depth_range(f, vp, z, X0, X1, Ylo, Yhi, za, zb)) break;
                if (!clip_span_depths(vp, k, tp.L, za, zb, Ylo, Yhi, X0, X1)) {
                    c0 = 1;
                    c1 = 0;
                    return;
                }
                c0 = max(c0, (int)floorf(ceilf(X0 - 0.5f) * (1.f / kTile)));
                c1 = min(c1, (int)floorf(floorf(X1 - 0.5f) * (1.f / kTile)));
            }
            return;
        }
        SubsetClip clip;
        make_clip_tab(vp, k, tp.L, z, clip);
        footprint_row_tiles_clipped(f, vp, ty, &clip, c0, c1);
    } else {
        footprint_row_tiles_clipped(f, vp, ty, nullptr, c0, c1);
    }
}

template <int kMulti = -1>
__device__ __forceinline__ void item_span(const Footprint& f, const ViewParams& vp, const TreeParams& tp,
                                          unsigned long long mask, int nsub, float z, int ty0, int rows, int it,
                                          int& ty, int& k, int& c0, int& c1) {
    item_locate(mask, ty0, rows, it, ty, k);
    item_cols<kMulti>(f, vp, tp, k, nsub, z, ty, c0, c1);
}

// A splat with at most this many (subset, row) items is counted and emitted by one
// thread; the others by a warp.
constexpr int kSplatThreadItems = 4;

// Items kept by the count for the emission.  A warp-counted splat j whose items fit in
// the list gets item_at[j] = its first entry there (kNoItems: not kept, the emission
// derives its items again); entry item_at[j] + it describes item it of the splat:
//   x = j, y = the item's first instance relative to the splat's first instance,
//   z = tile columns c0 | c1 << 16 (int16 each; (1, 0) when empty),
//   w = tile row | subset << 16;  x = kNoItems marks an entry that holds no item.
// The emission then writes every kept item without the footprint arithmetic, and count
// and emission agree by construction.
constexpr uint32_t kNoItems = 0xFFFFFFFFu;

__device__ __forceinline__ uint4 pack_item(uint32_t j, uint32_t first, int c0, int c1, int ty, int k) {
    if (c0 > c1) {
        c0 = 1;
        c1 = 0;
    }
    return make_uint4(j, first, (uint32_t)(uint16_t)(int16_t)c0 | ((uint32_t)(uint16_t)(int16_t)c1 << 16),
                      (uint32_t)ty | ((uint32_t)k << 16));
}

// Depth culling of the backward's instances: `cull` ([tiles, K] by view rank, nullptr:
// keep all) holds, per (tile, subset), the depth of the last splat the forward staged
// before every pixel of the tile was done in that subset (+inf if that never happened).
// A deeper instance cannot change any pixel, in the forward or in its replay.  `chunk`
// holds the (min, max) of `cull` over runs of kCullChunk tiles of a row, so most of a
// long span is kept or dropped without reading every tile.
constexpr int kCullChunk = 16;

__device__ __forceinline__ bool keep_tile(const float* __restrict__ cull, const ViewParams& vp, int ty, int c, int rank,
                                          float z) {
    return !cull || z <= cull[((size_t)ty * vp.tiles_x + c) * vp.K + rank];
}

__device__ __forceinline__ int cull_nchunk(const ViewParams& vp) { return (vp.tiles_x + kCullChunk - 1) / kCullChunk; }

// Entry of the chunk table for chunk ch of tile row ty in subset `rank`.
__device__ __forceinline__ size_t cull_chunk_index(const ViewParams& vp, int ty, int ch, int rank) {
    return ((size_t)ty * cull_nchunk(vp) + ch) * vp.K + rank;
}

// Whether the current binning group takes subsets of this view rank.
__device__ __forceinline__ bool rank_binned(const ViewParams& vp, int rank) {
    return rank >= vp.bin_lo && rank < vp.bin_hi;
}

// Whether tile (ty, c) is open in the group's open-tile table (which must be set).
__device__ __forceinline__ bool tile_open(const ViewParams& vp, int ty, int c) {
    const uint32_t* row = vp.open_prefix() + (size_t)ty * (vp.tiles_x + 1);
    return row[c + 1] != row[c];
}

// Tile columns [c0, c1] that bound every item span of the footprint (its ellipse and ball
// extents, widened by a pixel and a half against rounding).
__device__ __forceinline__ void footprint_tile_cols(const Footprint& f, const ViewParams& vp, int& c0, int& c1) {
    const float w = fminf(f.ex, f.bx) + 1.5f;
    c0 = (int)fmaxf(floorf((f.cx - w) * (1.f / kTile)), 0.f);
    c1 = (int)fminf(floorf((f.cx + w) * (1.f / kTile)), (float)(vp.tiles_x - 1));
}

// Whether the splat's tile box (rect: columns x..z, rows y..w) holds an open tile of the
// binning group (always, without an open-tile table).
__device__ __forceinline__ bool box_open(const ViewParams& vp, ushort4 r) {
    const uint32_t* sat = vp.open_sat();
    if (!sat) return true;
    if (r.x > r.z || r.y > r.w) return false;
    const size_t W1 = (size_t)vp.tiles_x + 1;
    const uint32_t n = sat[(r.w + 1) * W1 + r.z + 1] - sat[(size_t)r.y * W1 + r.z + 1] - sat[(r.w + 1) * W1 + r.x] +
                       sat[(size_t)r.y * W1 + r.x];
    return n != 0u;
}

// Number of tiles of [c0, c1] in row ty, ignoring the binning group, kept for a splat at
// depth z in subset `rank`.
__device__ __forceinline__ uint32_t kept_tiles_any_group(const float* __restrict__ cull,
                                                         const float2* __restrict__ chunk, const ViewParams& vp,
                                                         int ty, int c0, int c1, int rank, float z);

// Number of tiles of [c0, c1] in row ty kept for a splat at depth z in subset `rank`: in
// the binning group (rank range, open tiles), and not behind the depth table `cull`.  A
// group with an open-tile table is binned without a depth table.
__device__ __forceinline__ uint32_t kept_tiles(const float* __restrict__ cull, const float2* __restrict__ chunk,
                                               const ViewParams& vp, int ty, int c0, int c1, int rank, float z) {
    if (c0 > c1 || !rank_binned(vp, rank)) return 0u;
    const uint32_t* open = vp.open_prefix();
    if (open) {
        const uint32_t* row = open + (size_t)ty * (vp.tiles_x + 1);
        return row[c1 + 1] - row[c0];
    }
    return kept_tiles_any_group(cull, chunk, vp, ty, c0, c1, rank, z);
}

__device__ __forceinline__ uint32_t kept_tiles_any_group(const float* __restrict__ cull,
                                                         const float2* __restrict__ chunk, const ViewParams& vp,
                                                         int ty, int c0, int c1, int rank, float z) {
    if (c0 > c1) return 0u;
    if (!cull) return (uint32_t)(c1 - c0 + 1);
    uint32_t n = 0;
    for (int ch = c0 / kCullChunk; ch <= c1 / kCullChunk; ++ch) {
        const int lo = max(c0, ch * kCullChunk), hi = min(c1, ch * kCullChunk + kCullChunk - 1);
        const float2 mm = chunk[cull_chunk_index(vp, ty, ch, rank)];
        if (z > mm.y) continue;
        if (z <= mm.x) {
            n += (uint32_t)(hi - lo + 1);
            continue;
        }
        for (int c = lo; c <= hi; ++c) n += keep_tile(cull, vp, ty, c, rank, z);
    }
    return n;
}

// rank_of: the view rank of each subset (a copy in shared memory: lanes index it with
// different subsets).
__device__ __forceinline__ uint32_t item_tiles(const Footprint& f, const ViewParams& vp, const TreeParams& tp,
                                               const int8_t* rank_of, unsigned long long mask, int nsub, float z,
                                               int ty0, int rows, int it, const float* __restrict__ cull,
                                               const float2* __restrict__ chunk) {
    int ty, k, c0, c1;
    item_span(f, vp, tp, mask, nsub, z, ty0, rows, it, ty, k, c0, c1);
    return kept_tiles(cull, chunk, vp, ty, c0, c1, rank_of[k], z);
}

// Block-wide copy of the tree and the view's rank table into shared memory: the per-splat
// tree walks and per-item leaf paths index them with a different node or subset per lane,
// which kernel-parameter (constant) memory would serialise.  The whole block calls it.
__device__ __forceinline__ void stage_tree(const TreeParams& tp, const int8_t* rank_src, TreeParams& stp,
                                           int8_t* srank) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&tp);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&stp);
    for (int w = threadIdx.x; w < (int)(sizeof(TreeParams) / 4); w += blockDim.x) dst[w] = src[w];
    for (int k = threadIdx.x; k < 64; k += blockDim.x) srank[k] = rank_src[k];
    __syncthreads();
}

}  // namespace rgs
