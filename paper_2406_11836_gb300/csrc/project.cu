// Per-splat projection of Sec. 3.1 and its adjoint.
//
// Forward, one thread per splat: camera transform, near cull, EWA 2D covariance
// Sigma' = J W Sigma W^T J^T + dilation I (Jacobian linearisation of the pinhole model),
// conic and its Cholesky factor, SH colour at the viewing direction, sigmoid opacity,
// D_i = trunc_mult * max scale (Sec. 3.3), the conservative tile rectangle, the set of KD
// subsets N_k holding the splat (the D_i rule of Sec. 3.3) and the instance count.
//
// Precision.  A 4K frame puts projected centres at pixel coordinates up to ~4000, where
// one fp32 ulp is 2.4e-4 px, and the world->camera transform of a splat 30 units from
// the origin loses another ~1e-6 units; either alone moves a sub-pixel splat by more than
// the 1e-4 pixel tolerance allows.  The centre is therefore carried as an unevaluated
// sum hi + lo of two floats: the camera transform is a compensated dot product
// (error-free products and sums), and the perspective division and the intrinsics are
// done with error-free transformations too.  The blend kernels shift it to tile-relative
// coordinates once per instance.  The 2D covariance is formed as A A^T with A = J W R S,
// and its determinant by the Lagrange identity |A0|^2 |A1|^2 - (A0.A1)^2 = |A0 x A1|^2,
// so no cancellation occurs for elongated splats.  Everything else is plain fp32.
#include <cuda_fp16.h>

#include "eft.cuh"
#include "footprint.cuh"
#include "rgs_internal.cuh"

namespace rgs {
namespace {

// ------------------------------------------------------------------ real SH basis, degree <= 3
// Real spherical harmonics with the Condon-Shortley phase: for m != 0,
// Y_lm = sqrt(2) K_l|m| P_l^|m|(cos theta) {cos, sin}(|m| phi), K_lm^2 = (2l+1)/(4 pi) (l-m)!/(l+m)!,
// and r^l P_l^m(cos theta) e^{i m phi} written as polynomials of the unit direction.
constexpr double cx_sqrt(double x) {
    double r = x > 1 ? x : 1.0;
    for (int i = 0; i < 64; ++i) r = 0.5 * (r + x / r);
    return r;
}
constexpr double kPi = 3.14159265358979323846;
constexpr double fact(int n) { return n <= 1 ? 1.0 : n * fact(n - 1); }
constexpr double Klm(int l, int m) { return cx_sqrt((2 * l + 1) / (4 * kPi) * fact(l - m) / fact(l + m)); }
constexpr double S2 = 1.41421356237309504880;
// coefficient = normalisation times the leading integer of the Legendre polynomial
constexpr float c00 = (float)Klm(0, 0);
constexpr float c10 = (float)Klm(1, 0);             // z
constexpr float c11 = (float)(-S2 * Klm(1, 1));     // P_1^1 = -sin: -x, -y
constexpr float c20 = (float)(0.5 * Klm(2, 0));     // (3z^2 - 1)/2
constexpr float c21 = (float)(-3.0 * S2 * Klm(2, 1));  // P_2^1 = -3 sin cos: -3 xz, -3 yz
constexpr float c22 = (float)(3.0 * S2 * Klm(2, 2));   // P_2^2 = 3 sin^2: 3(x^2-y^2), 3*2xy
constexpr float c30 = (float)(0.5 * Klm(3, 0));        // (5z^3 - 3z)/2
constexpr float c31 = (float)(-1.5 * S2 * Klm(3, 1));  // P_3^1 = -3/2 (5z^2-1) sin
constexpr float c32 = (float)(15.0 * S2 * Klm(3, 2));  // P_3^2 = 15 sin^2 cos
constexpr float c33 = (float)(-15.0 * S2 * Klm(3, 3)); // P_3^3 = -15 sin^3

// Basis values Y[k] (k = l*l + m + l) and, when dY != nullptr, their gradients as
// polynomials of (x, y, z).
template <int DEG>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float* Y, float3* dY) {
    Y[0] = c00;
    if (dY) dY[0] = make_float3(0.f, 0.f, 0.f);
    if (DEG >= 1) {
        Y[1] = c11 * y;  // m = -1
        Y[2] = c10 * z;  // m = 0
        Y[3] = c11 * x;  // m = 1
        if (dY) {
            dY[1] = make_float3(0.f, c11, 0.f);
            dY[2] = make_float3(0.f, 0.f, c10);
            dY[3] = make_float3(c11, 0.f, 0.f);
        }
    }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = c22 * 2.f * x * y;                     // m = -2
        Y[5] = c21 * y * z;                           // m = -1
        Y[6] = c20 * (3.f * zz - (xx + yy + zz));     // m = 0: 3z^2 - r^2
        Y[7] = c21 * x * z;                           // m = 1
        Y[8] = c22 * (xx - yy);                       // m = 2
        if (dY) {
            dY[4] = make_float3(c22 * 2.f * y, c22 * 2.f * x, 0.f);
            dY[5] = make_float3(0.f, c21 * z, c21 * y);
            dY[6] = make_float3(-2.f * c20 * x, -2.f * c20 * y, 4.f * c20 * z);
            dY[7] = make_float3(c21 * z, 0.f, c21 * x);
            dY[8] = make_float3(2.f * c22 * x, -2.f * c22 * y, 0.f);
        }
    }
    if (DEG >= 3) {
        float xx = x * x, yy = y * y, zz = z * z;
        float q = 5.f * zz - (xx + yy + zz);          // 5 z^2 - r^2
        Y[9] = c33 * (3.f * xx * y - yy * y);         // m = -3: Im (x+iy)^3
        Y[10] = c32 * 2.f * x * y * z;                // m = -2
        Y[11] = c31 * y * q;                          // m = -1
        Y[12] = c30 * z * (5.f * zz - 3.f * (xx + yy + zz));  // m = 0
        Y[13] = c31 * x * q;                          // m = 1
        Y[14] = c32 * z * (xx - yy);                  // m = 2
        Y[15] = c33 * (xx * x - 3.f * x * yy);        // m = 3: Re (x+iy)^3
        if (dY) {
            dY[9] = make_float3(c33 * 6.f * x * y, c33 * (3.f * xx - 3.f * yy), 0.f);
            dY[10] = make_float3(c32 * 2.f * y * z, c32 * 2.f * x * z, c32 * 2.f * x * y);
            dY[11] = make_float3(c31 * y * (-2.f * x), c31 * (q - 2.f * yy), c31 * y * 8.f * z);
            dY[12] = make_float3(c30 * z * (-6.f * x), c30 * z * (-6.f * y), c30 * (15.f * zz - 3.f * (xx + yy + zz) - 6.f * zz));
            dY[13] = make_float3(c31 * (q - 2.f * xx), c31 * x * (-2.f * y), c31 * x * 8.f * z);
            dY[14] = make_float3(c32 * 2.f * x * z, -c32 * 2.f * y * z, c32 * (xx - yy));
            dY[15] = make_float3(c33 * (3.f * xx - 3.f * yy), c33 * (-6.f * x * y), 0.f);
        }
    }
}

// ------------------------------------------------------------------ rotation from a quaternion
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// Subsets holding a splat: leaves of the KD tree whose box, dilated by D in every axis,
// contains mu (left branch: mu[a] - D < s, right branch: mu[a] + D >= s).  Iterative DFS.
__device__ __forceinline__ unsigned long long subset_mask(const TreeParams& tp, float mx, float my, float mz, float D) {
    // level by level: `cur` holds the reachable nodes of the level (bit i: node 2^d - 1 + i)
    unsigned long long cur = 1ull;
    for (int d = 0; d < tp.L; ++d) {
        unsigned long long next = 0ull, m = cur;
        const int first = (1 << d) - 1;
        while (m) {
            const int i = __ffsll((long long)m) - 1;
            m &= m - 1;
            const int j = first + i;
            const int a = tp.axis[j];
            const float s = tp.split[j];
            const float c = a == 0 ? mx : (a == 1 ? my : mz);
            if (c - D < s) next |= 1ull << (2 * i);
            if (c + D >= s) next |= 1ull << (2 * i + 1);
        }
        cur = next;
    }
    return cur;
}

// The splat's colour before the clamp, raw_c = sum_k sh[k][c] Y_k + 1/2 (coefficients
// k-major, RGB inner).  kVec: the coefficients are read as float4 (their block is 16-byte
// aligned); the per-channel accumulation order is the same either way.
template <int NSH, bool kVec>
__device__ __forceinline__ void sh_colour(const float* __restrict__ sh, const float* Y, float raw[3]) {
    raw[0] = raw[1] = raw[2] = 0.5f;
    if constexpr (kVec) {
        const float4* s4 = reinterpret_cast<const float4*>(sh);
#pragma unroll
        for (int q = 0; q < NSH * 3 / 4; ++q) {
            const float4 v = __ldg(s4 + q);
            const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int idx = 4 * q + t;
                raw[idx % 3] = fmaf(e[t], Y[idx / 3], raw[idx % 3]);
            }
        }
    } else {
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int k = 0; k < NSH; ++k) raw[c] = fmaf(sh[3 * k + c], Y[k], raw[c]);
        }
    }
}

struct SplatIn {
    float mu[3], ls[3], q[4], logit;
};

__device__ __forceinline__ void load_splat(const rgs_gaussians& g, int64_t i, SplatIn& s) {
    s.mu[0] = g.means[3 * i]; s.mu[1] = g.means[3 * i + 1]; s.mu[2] = g.means[3 * i + 2];
    s.ls[0] = g.log_scales[3 * i]; s.ls[1] = g.log_scales[3 * i + 1]; s.ls[2] = g.log_scales[3 * i + 2];
    float4 q = reinterpret_cast<const float4*>(g.quats)[i];
    s.q[0] = q.x; s.q[1] = q.y; s.q[2] = q.z; s.q[3] = q.w;
    s.logit = g.opacity_logits[i];
}

// Camera-space centre with the compensated transform; returns z (hi) and the projected
// centre as hi + lo pairs.
__device__ __forceinline__ void project_centre(const ViewParams& vp, const float mu[3], float p[3], float& mxh,
                                               float& mxl, float& myh, float& myl, float* z_lo = nullptr) {
    float xh, xl, yh, yl, zh, zl;
    dot3_plus(vp.R[0], mu[0], vp.R[1], mu[1], vp.R[2], mu[2], vp.t[0], xh, xl);
    dot3_plus(vp.R[3], mu[0], vp.R[4], mu[1], vp.R[5], mu[2], vp.t[1], yh, yl);
    dot3_plus(vp.R[6], mu[0], vp.R[7], mu[1], vp.R[8], mu[2], vp.t[2], zh, zl);
    p[0] = xh; p[1] = yh; p[2] = zh;
    if (z_lo) *z_lo = zl;
    // u = x/z to about two floats: q + (x - q z)/z
    float qx = __fdiv_rn(xh, zh);
    float rx = __fmaf_rn(-qx, zh, xh);
    rx = __fadd_rn(rx, __fsub_rn(xl, __fmul_rn(qx, zl)));
    float qxl = __fdiv_rn(rx, zh);
    float qy = __fdiv_rn(yh, zh);
    float ry = __fmaf_rn(-qy, zh, yh);
    ry = __fadd_rn(ry, __fsub_rn(yl, __fmul_rn(qy, zl)));
    float qyl = __fdiv_rn(ry, zh);
    // mean = f * u + c
    float m, e, s, t;
    two_prod(vp.fx, qx, m, e);
    e = __fmaf_rn(vp.fx, qxl, e);
    two_sum(m, vp.cx, s, t);
    fast_two_sum(s, __fadd_rn(e, t), mxh, mxl);
    two_prod(vp.fy, qy, m, e);
    e = __fmaf_rn(vp.fy, qyl, e);
    two_sum(m, vp.cy, s, t);
    fast_two_sum(s, __fadd_rn(e, t), myh, myl);
}

// Shared forward intermediates (recomputed by the backward).
struct Proj {
    float p[3], z, u, v;       // camera-space centre, u = x/z, v = y/z
    float s[3], Rq[9], qn[4], qnorm;
    float T0[3], T1[3];        // T = J W
    float A0[3], A1[3];        // A = T R_q S
    float sxx, sxy, syy, det;  // Sigma' and its determinant
    float ca, cb, cc;          // conic
    float alpha;
};

__device__ __forceinline__ void ewa(const ViewParams& vp, const SplatIn& si, const float p[3], Proj& P) {
    P.p[0] = p[0]; P.p[1] = p[1]; P.p[2] = p[2];
    P.z = p[2];
    float iz = 1.f / P.z;
    P.u = p[0] * iz;
    P.v = p[1] * iz;
    float qn2 = si.q[0] * si.q[0] + si.q[1] * si.q[1] + si.q[2] * si.q[2] + si.q[3] * si.q[3];
    P.qnorm = sqrtf(qn2);
    float iq = 1.f / P.qnorm;
    for (int j = 0; j < 4; ++j) P.qn[j] = si.q[j] * iq;
    quat_rot(P.qn[0], P.qn[1], P.qn[2], P.qn[3], P.Rq);
    for (int j = 0; j < 3; ++j) P.s[j] = __expf(si.ls[j]);
    // T = J W: rows (fx/z)(W0 - u W2), (fy/z)(W1 - v W2)
    float ax = vp.fx * iz, ay = vp.fy * iz;
    for (int c = 0; c < 3; ++c) {
        P.T0[c] = ax * (vp.R[c] - P.u * vp.R[6 + c]);
        P.T1[c] = ay * (vp.R[3 + c] - P.v * vp.R[6 + c]);
    }
    // A = T Rq diag(s)
    for (int c = 0; c < 3; ++c) {
        float r0 = P.T0[0] * P.Rq[c] + P.T0[1] * P.Rq[3 + c] + P.T0[2] * P.Rq[6 + c];
        float r1 = P.T1[0] * P.Rq[c] + P.T1[1] * P.Rq[3 + c] + P.T1[2] * P.Rq[6 + c];
        P.A0[c] = r0 * P.s[c];
        P.A1[c] = r1 * P.s[c];
    }
    float n0 = P.A0[0] * P.A0[0] + P.A0[1] * P.A0[1] + P.A0[2] * P.A0[2];
    float n1 = P.A1[0] * P.A1[0] + P.A1[1] * P.A1[1] + P.A1[2] * P.A1[2];
    float d01 = P.A0[0] * P.A1[0] + P.A0[1] * P.A1[1] + P.A0[2] * P.A1[2];
    float cx = P.A0[1] * P.A1[2] - P.A0[2] * P.A1[1];
    float cy = P.A0[2] * P.A1[0] - P.A0[0] * P.A1[2];
    float cz = P.A0[0] * P.A1[1] - P.A0[1] * P.A1[0];
    float dl = vp.dilation;
    P.sxx = n0 + dl;
    P.syy = n1 + dl;
    P.sxy = d01;
    P.det = (cx * cx + cy * cy + cz * cz) + dl * (n0 + n1) + dl * dl;
    float idet = 1.f / P.det;
    P.ca = P.syy * idet;
    P.cb = -P.sxy * idet;
    P.cc = P.sxx * idet;
    P.alpha = 1.f / (1.f + __expf(-si.logit));
}

// Depth below the resolution of the float z = zh + zl (|zl| <= ulp(zh)/2): zl in units of
// ulp(zh)/2^16, offset to [0, 2^16).  Sorting by this and then stably by the bits of zh
// orders splats by z to about 2^-39 relative, so that splats whose depths round to the
// same float still blend in the order of their exact depths.
__device__ __forceinline__ uint32_t depth_fraction(float zh, float zl) {
    const uint32_t e = (__float_as_uint(zh) >> 23) & 0xffu;
    if (e < 24u) return 32768u;                                     // zh below 2^-103: no fraction
    const float inv_ulp = __uint_as_float((277u - e) << 23);        // 2^(150 - e) = 1 / ulp(zh)
    const int q = __float2int_rn(zl * inv_ulp * 65536.f) + 32768;  // exact power-of-two scalings
    return (uint32_t)min(max(q, 0), 65535);
}

// ------------------------------------------------------------------ forward kernel
constexpr int kWarpCountItems = kSplatThreadItems;   // splats with more items are counted by the whole warp

// Projection of splat i (valid: i < n) into one view.  Outputs go to index j of the
// per-splat arrays of b; the instance and visible-splat totals are added to counters[0..1]
// and, when non-null, slot_counters[0..1].  Every lane of the warp must call it.  kFoot:
// the foot reading of x_i (its ball region, side array and depth interval).
template <int DEG, bool kVecSH, bool kFoot = false>
__device__ __forceinline__ void project_fwd_body(const rgs_gaussians& g, int64_t i, bool valid, const ViewParams& vp,
                                                 const TreeParams& tp, const int8_t* rank_of, const RasterBuffers& b,
                                                 int64_t j, unsigned long long* counters,
                                                 unsigned long long* slot_counters,
                                                 unsigned long long* blk_tot = nullptr) {
    constexpr int NSH = (DEG + 1) * (DEG + 1);
    const int lane = threadIdx.x & 31;
    // candidate state handed to the counting phase
    bool cand = false;
    float mxh = 0.f, myh = 0.f, l11 = 0.f, l12 = 0.f, l22 = 0.f, alpha = 0.f, rho2 = 0.f, z = 0.f, zr = 0.f;
    unsigned long long mask = 0;
    int ty0 = 0, ty1 = -1, tx0 = 0, tx1 = 0, nsub = 0;
    if (valid) {
        SplatIn si;
        load_splat(g, i, si);
        float p[3], mxl, myl, zl;
        project_centre(vp, si.mu, p, mxh, mxl, myh, myl, &zl);
        z = p[2];
        const float smax = fmaxf(si.ls[0], fmaxf(si.ls[1], si.ls[2]));
        const float D = vp.trunc_mult * __expf(smax);
        alpha = 1.f / (1.f + __expf(-si.logit));
        // A splat contributes nowhere unless z > near and alpha >= alpha_min, nor outside the
        // ball test's screen ellipse (semi-axes f D / z around the centre; widened by 0.1%
        // and a pixel against rounding), so splats whose ellipse misses the image skip the
        // EWA projection.
        float rball = D / z;   // ball radius in normalised image units
        if (kFoot) {
            // foot reading: the rays passing within D of the centre form a cone of half-angle
            // al = asin(D / |p|) around p, whose axis makes th with the optical axis.  A
            // direction within al of p lands within al / cos^2(th + al) of the projected
            // centre (the gnomonic map stretches arcs by at most 1 / cos^2 of their polar
            // angle), so that disc, widened by 1%, bounds every pixel the ball test accepts;
            // from th + al = 89 degrees on it is taken as unbounded.
            const float pxy2 = fmaf(p[0], p[0], p[1] * p[1]);
            const float pr2 = fmaf(z, z, pxy2);
            rball = __int_as_float(0x7f800000);
            if (D * D < pr2) {
                // cos(th + al) = (z sqrt(|p|^2 - D^2) - sqrt(x^2 + y^2) D) / |p|^2
                const float c = (z * sqrtf(pr2 - D * D) - sqrtf(pxy2) * D) / pr2;
                if (c > 0.0175f) rball = asinf(D * rsqrtf(pr2)) / (c * c) * 1.01f + 1e-7f;
            }
        }
        const float bxr = vp.fx * rball * 1.001f + 1.f, byr = vp.fy * rball * 1.001f + 1.f;
        const bool on_screen = mxh + bxr >= 0.f && mxh - bxr <= (float)vp.W && myh + byr >= 0.f &&
                               myh - byr <= (float)vp.H;
        if (z > vp.near_z && alpha >= vp.alpha_min && isfinite(mxh) && isfinite(myh) && on_screen) {
            Proj P;
            ewa(vp, si, p, P);
            l11 = sqrtf(P.ca);
            l12 = P.cb / l11;
            l22 = rsqrtf(P.det * P.ca);
            const float rb = D / z;                   // ball radius in normalised image units
            mask = subset_mask(tp, si.mu[0], si.mu[1], si.mu[2], D);
            nsub = __popcll(mask);
            // foot reading: the record carries the disc bounding the foot's ball region
            // (footprints, counts and emission use it as they use the depth plane's ball),
            // and the ball radius itself moves to a side array for the per-pixel test
            rho2 = nsub > 1 ? -(rball * rball) : rball * rball;
            if (kFoot) zr = foot_depth_radius(z, rb * rb);
            if (isfinite(P.det) && P.det > 0.f && isfinite(l11) && isfinite(l22)) {
                const Footprint f = make_footprint(mxh, myh, l11, l12, l22, alpha, rho2, vp);
                footprint_tile_rows(f, vp, ty0, ty1);
                footprint_tile_cols(f, vp, tx0, tx1);
                cand = ty0 <= ty1;
            }
            if (cand) {
                // colour at dir = normalise(mu - o)
                float dx = si.mu[0] - vp.o[0], dy = si.mu[1] - vp.o[1], dz = si.mu[2] - vp.o[2];
                float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
                float Y[16];
                sh_eval<DEG>(dx * inv, dy * inv, dz * inv, Y, nullptr);
                float rgb[3];
                sh_colour<NSH, kVecSH>(g.sh + i * NSH * 3, Y, rgb);
                for (int c = 0; c < 3; ++c) rgb[c] = fmaxf(rgb[c], 0.f);
                __half2 lo = __floats2half2_rn(mxl, myl);
                float lo_bits = __uint_as_float(*reinterpret_cast<uint32_t*>(&lo));
                b.rec[3 * j] = make_float4(mxh, myh, lo_bits, alpha);
                b.rec[3 * j + 1] = make_float4(l11, l12, l22, rho2);
                b.rec[3 * j + 2] = make_float4(rgb[0], rgb[1], rgb[2], z);
                if (kFoot) b.foot_side[j] = make_float4(rb * rb, zl, mxl, myl);
                b.rect[j] = make_ushort4((unsigned short)tx0, (unsigned short)ty0, (unsigned short)tx1,
                                         (unsigned short)ty1);
                b.mask[j] = mask;
                b.dkey[j] = __float_as_uint(z);   // z > 0: the bit pattern sorts like the value
                b.dkey_lo[j] = depth_fraction(z, zl);
            }
        }
    }
    // ---- count the tile instances: small splats per thread, large ones per warp
    const int rows = ty1 - ty0 + 1;
    const int items = cand ? nsub * rows : 0;
    // count: every instance (visibility and capacity); count_bin: those of the first
    // binning group (its ranks; no open-tile table is set before the first blend)
    uint32_t count = 0, count_bin = 0;
    if (cand && items <= kWarpCountItems) {
        Footprint f = make_footprint(mxh, myh, l11, l12, l22, alpha, rho2, vp);
        f.zr = zr;
        for (int it = 0; it < items; ++it) {
            int ty, k, c0, c1;
            item_span(f, vp, tp, mask, nsub, z, ty0, rows, it, ty, k, c0, c1);
            const uint32_t w = kept_tiles_any_group(b.cull, b.cull_chunk, vp, ty, c0, c1, rank_of[k], z);
            count += w;
            count_bin += rank_binned(vp, rank_of[k]) ? w : 0u;
        }
    }
    unsigned big = __ballot_sync(0xffffffffu, items > kWarpCountItems);
    uint32_t span_at = kNoItems;
    // one reservation of item-list entries for all the warp's large splats: lane l's
    // entries start at res + (the large splats' items in lanes below l)
    unsigned long long res = 0;
    uint32_t res_pre = 0;
    if (big && b.items) {
        uint32_t mine = items > kWarpCountItems ? (uint32_t)items : 0u, incl = mine;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        res_pre = incl - mine;
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        if (lane == 0) res = atomicAdd(b.item_ctr, (unsigned long long)tot);
        res = __shfl_sync(0xffffffffu, res, 0);
    }
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const float fx_ = __shfl_sync(0xffffffffu, mxh, src), fy_ = __shfl_sync(0xffffffffu, myh, src);
        const float a_ = __shfl_sync(0xffffffffu, l11, src), b_ = __shfl_sync(0xffffffffu, l12, src);
        const float c_ = __shfl_sync(0xffffffffu, l22, src), al_ = __shfl_sync(0xffffffffu, alpha, src);
        const float r_ = __shfl_sync(0xffffffffu, rho2, src), z_ = __shfl_sync(0xffffffffu, z, src);
        const unsigned long long m_ = __shfl_sync(0xffffffffu, mask, src);
        const int t0_ = __shfl_sync(0xffffffffu, ty0, src), rows_ = __shfl_sync(0xffffffffu, rows, src);
        const int items_ = __shfl_sync(0xffffffffu, items, src);
        Footprint f = make_footprint(fx_, fy_, a_, b_, c_, al_, r_, vp);
        f.zr = __shfl_sync(0xffffffffu, zr, src);
        const int ns = __popcll(m_);
        const uint32_t j_ = (uint32_t)__shfl_sync(0xffffffffu, (uint32_t)j, src);
        // keep the items for the emission when the list has room (item_ctr counts the
        // entries taken, reserved once per warp; the one splat whose entries cross the end
        // voids its part inside)
        uint32_t sb = kNoItems;
        if (b.items) {
            const unsigned long long s0 = res + (unsigned long long)__shfl_sync(0xffffffffu, res_pre, src);
            if (s0 + (unsigned long long)items_ <= b.item_cap) {
                sb = (uint32_t)s0;
            } else {
                for (unsigned long long q = s0 + (unsigned long long)lane; q < b.item_cap; q += 32)
                    b.items[q] = make_uint4(kNoItems, 0u, 0u, 0u);
            }
        }
        // the records hold each item's first instance among the first group's instances
        uint32_t acc = 0, acc_bin = 0;   // instances of the rounds before
        for (int it0 = 0; it0 < items_; it0 += 32) {
            const int it = it0 + lane;
            int ty = 0, k = 0, c0 = 1, c1 = 0;
            uint32_t w = 0, wb = 0;
            if (it < items_) {
                item_span(f, vp, tp, m_, ns, z_, t0_, rows_, it, ty, k, c0, c1);
                w = kept_tiles_any_group(b.cull, b.cull_chunk, vp, ty, c0, c1, rank_of[k], z_);
                wb = rank_binned(vp, rank_of[k]) ? w : 0u;
            }
            uint32_t incl = wb, incl_all = w;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                const uint32_t ya = __shfl_up_sync(0xffffffffu, incl_all, o);
                if (lane >= o) {
                    incl += y;
                    incl_all += ya;
                }
            }
            if (sb != kNoItems && it < items_) {
                b.items[sb + it] = pack_item(j_, acc_bin + incl - wb, c0, c1, ty, k);
                if (b.item_first_all) b.item_first_all[sb + it] = acc + incl_all - w;
            }
            acc_bin += __shfl_sync(0xffffffffu, incl, 31);
            acc += __shfl_sync(0xffffffffu, incl_all, 31);
        }
        if (lane == src) {
            count = acc;
            count_bin = acc_bin;
            span_at = sb;
        }
    }
    if (valid) b.cnt[j] = count;
    if (valid && b.cnt_bin) b.cnt_bin[j] = count_bin;
    if (valid && b.item_at && items > kWarpCountItems) b.item_at[j] = span_at;
    // totals: instances and visible splats
    unsigned long long c64 = count;
    unsigned vis_n = count > 0;
    for (int o = 16; o > 0; o >>= 1) {
        c64 += __shfl_xor_sync(0xffffffffu, c64, o);
        vis_n += __shfl_xor_sync(0xffffffffu, vis_n, o);
    }
    // blk_tot (shared, nullable): the block's totals (instances, visible splats, first-group
    // instances), added to the counters once per block by the caller
    if (b.cnt_bin) {
        unsigned long long cb = count_bin;
        for (int o = 16; o > 0; o >>= 1) cb += __shfl_xor_sync(0xffffffffu, cb, o);
        if (lane == 0 && cb) atomicAdd(blk_tot ? &blk_tot[2] : b.bin_ctr, cb);   // the first group's instances
    }
    if (lane == 0 && (c64 | vis_n)) {
        if (blk_tot) {   // the caller adds them to counters (and the slot's) once per block
            atomicAdd(&blk_tot[0], c64);
            atomicAdd(&blk_tot[1], (unsigned long long)vis_n);
        } else {
            atomicAdd(&counters[0], c64);
            atomicAdd(&counters[1], (unsigned long long)vis_n);
            if (slot_counters) {
                atomicAdd(&slot_counters[0], c64);
                atomicAdd(&slot_counters[1], (unsigned long long)vis_n);
            }
        }
    }
}

template <int DEG, bool kVecSH, bool kFoot>
__global__ void __launch_bounds__(256, 3)
project_fwd_kernel(rgs_gaussians g, ViewParams vp, TreeParams tp, RasterBuffers b) {
    __shared__ TreeParams stp;
    __shared__ int8_t srank[64];
    stage_tree(tp, vp.rank_of, stp, srank);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    project_fwd_body<DEG, kVecSH, kFoot>(g, i, i < g.n, vp, stp, srank, b, i, b.counters, nullptr);
}

// Screen cull before the projection: a splat stays a candidate unless it is certainly
// culled by the projection's own tests (behind the near plane, alpha below alpha_min, or
// its ball-test ellipse off the image), judged in plain fp32 with margins that cover the
// difference to the compensated centre: 1e-4 of the near depth, 1% of the ellipse's
// semi-axes plus 2 pixels.  Alpha is computed exactly as the projection computes it.
// Candidates are appended to `cand` (counters[13]); every other splat gets cnt = 0.
// The projection then runs on full warps of candidates.
__device__ __forceinline__ bool screen_keep(const rgs_gaussians& g, const ViewParams& vp, int64_t i) {
    const float mx = g.means[3 * i], my = g.means[3 * i + 1], mz = g.means[3 * i + 2];
    const float ls = fmaxf(g.log_scales[3 * i], fmaxf(g.log_scales[3 * i + 1], g.log_scales[3 * i + 2]));
    const float alpha = 1.f / (1.f + __expf(-g.opacity_logits[i]));
    const float x = fmaf(vp.R[0], mx, fmaf(vp.R[1], my, fmaf(vp.R[2], mz, vp.t[0])));
    const float y = fmaf(vp.R[3], mx, fmaf(vp.R[4], my, fmaf(vp.R[5], mz, vp.t[1])));
    const float z = fmaf(vp.R[6], mx, fmaf(vp.R[7], my, fmaf(vp.R[8], mz, vp.t[2])));
    bool keep = alpha >= vp.alpha_min && !(z < vp.near_z * (1.f - 1e-4f));
    if (keep && z > 0.f) {
        const float rball = vp.trunc_mult * __expf(ls) / z;
        const float cxp = fmaf(vp.fx, x / z, vp.cx), cyp = fmaf(vp.fy, y / z, vp.cy);
        const float bx = (vp.fx * rball * 1.001f + 1.f) * 1.01f + 2.f, by = (vp.fy * rball * 1.001f + 1.f) * 1.01f + 2.f;
        // off screen only when every comparison is certain (NaN and inf stay candidates)
        if (cxp + bx < 0.f || cxp - bx > (float)vp.W || cyp + by < 0.f || cyp - by > (float)vp.H) keep = false;
    }
    return keep;
}

// Four splats per thread (a block covers kCullPerBlock consecutive splats) and one append
// per block: one atomic per warp on the single candidate counter serialised the pass.
constexpr int kCullPerThread = 4;
constexpr int kCullPerBlock = 256 * kCullPerThread;
__global__ void __launch_bounds__(256)
screen_cull_kernel(rgs_gaussians g, ViewParams vp, uint32_t* __restrict__ cnt, uint32_t* __restrict__ cand,
                   unsigned long long* __restrict__ counters) {
    __shared__ uint32_t s_off[8];
    __shared__ unsigned long long s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * kCullPerBlock + threadIdx.x;
    unsigned bal[kCullPerThread];
    uint32_t wn = 0;
#pragma unroll
    for (int k = 0; k < kCullPerThread; ++k) {
        const int64_t i = i0 + 256 * k;
        const bool keep = i < g.n && screen_keep(g, vp, i);
        if (i < g.n && !keep) cnt[i] = 0u;
        bal[k] = __ballot_sync(0xffffffffu, keep);
        wn += __popc(bal[k]);
    }
    if (lane == 0) s_off[warp] = wn;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int w = 0; w < 8; ++w) {
            const uint32_t c = s_off[w];
            s_off[w] = run;
            run += c;
        }
        s_base = run ? atomicAdd(&counters[13], (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    unsigned long long pos = s_base + s_off[warp];
    const unsigned lower = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < kCullPerThread; ++k) {
        if ((bal[k] >> lane) & 1u) cand[pos + __popc(bal[k] & lower)] = (uint32_t)(i0 + 256 * k);
        pos += __popc(bal[k]);
    }
}

// The screen cull of a batch: block x tests splats [kCullPerBlock (x / kMaxSlots),
// +kCullPerBlock) against the view of slot x % kMaxSlots and appends the candidates to the
// slot's list (vis_pos from slot * N on, counted in counters[kBatchCandCounters + slot]),
// once per block.
__global__ void __launch_bounds__(256)
screen_cull_batch_kernel(rgs_gaussians g, const BatchSlot* __restrict__ slots, const BatchHeader* __restrict__ hdr,
                         uint32_t* __restrict__ cnt, uint32_t* __restrict__ cand,
                         unsigned long long* __restrict__ counters) {
    const int slot = blockIdx.x % kMaxSlots;
    if (slot >= hdr->S) return;   // uniform across the block
    __shared__ ViewParams svp;
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&slots[slot].vp);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&svp);
        for (int w = threadIdx.x; w < (int)(sizeof(ViewParams) / 4); w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ uint32_t s_off[8];
    __shared__ unsigned long long s_base;
    const int64_t i0 = (int64_t)(blockIdx.x / kMaxSlots) * kCullPerBlock + threadIdx.x;
    unsigned bal[kCullPerThread];
    uint32_t wn = 0;
#pragma unroll
    for (int k = 0; k < kCullPerThread; ++k) {
        const int64_t i = i0 + 256 * k;
        const bool keep = i < g.n && screen_keep(g, svp, i);
        if (i < g.n && !keep) cnt[(int64_t)slot * g.n + i] = 0u;
        bal[k] = __ballot_sync(0xffffffffu, keep);
        wn += __popc(bal[k]);
    }
    if (lane == 0) s_off[warp] = wn;
    __syncthreads();
    if (threadIdx.x == 0) {   // one append per block
        uint32_t run = 0;
        for (int w = 0; w < 8; ++w) {
            const uint32_t c = s_off[w];
            s_off[w] = run;
            run += c;
        }
        s_base = run ? atomicAdd(&counters[kBatchCandCounters + slot], (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    uint32_t* list = cand + (int64_t)slot * g.n;
    unsigned long long pos = s_base + s_off[warp];
    const unsigned lower = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < kCullPerThread; ++k) {
        if ((bal[k] >> lane) & 1u) list[pos + __popc(bal[k] & lower)] = (uint32_t)(i0 + 256 * k);
        pos += __popc(bal[k]);
    }
}

// The projection over the candidates of screen_cull_kernel, one per thread; the grid
// covers every splat and the blocks past the candidate count (read from the device) end
// at once.
template <int DEG, bool kVecSH>
__global__ void __launch_bounds__(256, 3)
project_cand_kernel(rgs_gaussians g, ViewParams vp, TreeParams tp, RasterBuffers b, const uint32_t* __restrict__ cand) {
    __shared__ TreeParams stp;
    __shared__ int8_t srank[64];
    const unsigned long long nc = b.counters[13];
    const unsigned long long c = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if ((unsigned long long)blockIdx.x * blockDim.x >= nc) return;   // uniform across the block
    __shared__ unsigned long long s_tot[3];   // instances, visible splats, first-group instances
    if (threadIdx.x < 3) s_tot[threadIdx.x] = 0ull;
    stage_tree(tp, vp.rank_of, stp, srank);   // (its barrier also orders the zeroing)
    const bool valid = c < nc;
    const int64_t i = valid ? (int64_t)cand[c] : 0;
    project_fwd_body<DEG, kVecSH, false>(g, i, valid, vp, stp, srank, b, i, b.counters, nullptr, s_tot);
    __syncthreads();
    if (threadIdx.x == 0) {   // one atomic per counter and block: per warp they serialised
        if (s_tot[0] | s_tot[1]) {
            atomicAdd(&b.counters[0], s_tot[0]);
            atomicAdd(&b.counters[1], s_tot[1]);
        }
        if (s_tot[2]) atomicAdd(b.bin_ctr, s_tot[2]);
    }
}

// The batch projection over each slot's screen-cull candidates: block x takes candidates
// [256 (x / kMaxSlots), +256) of slot x % kMaxSlots; blocks past the slot's count end at once.
template <int DEG, bool kVecSH>
__global__ void __launch_bounds__(256, 3)
project_cand_batch_kernel(rgs_gaussians g, const BatchSlot* __restrict__ slots, const BatchHeader* __restrict__ hdr,
                          TreeParams tp, RasterBuffers b, unsigned long long* __restrict__ counters) {
    const int slot = blockIdx.x % kMaxSlots;
    if (slot >= hdr->S) return;   // uniform across the block
    const unsigned long long nc = counters[kBatchCandCounters + slot];
    const unsigned long long c0 = (unsigned long long)(blockIdx.x / kMaxSlots) * blockDim.x;
    if (c0 >= nc) return;
    __shared__ ViewParams svp;
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&slots[slot].vp);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&svp);
        for (int w = threadIdx.x; w < (int)(sizeof(ViewParams) / 4); w += blockDim.x) dst[w] = src[w];
    }
    __shared__ TreeParams stp;
    __shared__ int8_t srank[64];
    stage_tree(tp, slots[slot].vp.rank_of, stp, srank);   // its barrier also publishes svp
    const unsigned long long c = c0 + threadIdx.x;
    const bool valid = c < nc;
    const int64_t i = valid ? (int64_t)b.vis_pos[(int64_t)slot * g.n + (int64_t)c] : 0;
    __shared__ unsigned long long s_tot[3];
    if (threadIdx.x < 3) s_tot[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned long long* slot_counters = counters + kBatchSlotCounters + 2 * slot;
    project_fwd_body<DEG, kVecSH>(g, i, valid, svp, stp, srank, b, (int64_t)slot * g.n + i, counters, slot_counters,
                                  s_tot);
    __syncthreads();
    if (threadIdx.x == 0) {   // the block's totals, once (every splat of the block is in this slot)
        if (s_tot[0] | s_tot[1]) {
            atomicAdd(&counters[0], s_tot[0]);
            atomicAdd(&counters[1], s_tot[1]);
            atomicAdd(&slot_counters[0], s_tot[0]);
            atomicAdd(&slot_counters[1], s_tot[1]);
        }
        if (s_tot[2]) atomicAdd(b.bin_ctr, s_tot[2]);
    }
}

// ------------------------------------------------------------------ backward kernel
// Pulls the per-splat 2D gradients (mean, conic, alpha, colour) back to the parameters:
// colour -> SH coefficients and viewing direction; conic -> Sigma' -> A = J W Rq S ->
// (J, Rq, S); J and the mean -> camera-space centre -> world centre; Rq -> normalised
// quaternion -> quaternion; S -> log-scales; alpha -> logit.  Gradients are added to the
// caller's buffers; one thread owns one splat, so no atomics are needed.
template <int DEG, bool kVecSH>
__global__ void __launch_bounds__(128)
project_bwd_kernel(rgs_gaussians g, rgs_gaussian_grads gr, ViewParams vp, const float4* __restrict__ g2d) {
    constexpr int NSH = (DEG + 1) * (DEG + 1);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    float4 ga = g2d[3 * i], gb = g2d[3 * i + 1], gc = g2d[3 * i + 2];
    if (ga.x == 0.f && ga.y == 0.f && ga.z == 0.f && ga.w == 0.f && gb.x == 0.f && gb.y == 0.f && gb.z == 0.f &&
        gb.w == 0.f && gc.x == 0.f)
        return;
    const float g_mx = ga.x, g_my = ga.y, g_ca = ga.z, g_cb = ga.w, g_cc = gb.x, g_alpha = gb.y;
    const float g_rgb[3] = {gb.z, gb.w, gc.x};

    SplatIn si;
    load_splat(g, i, si);
    float p[3], mxh, mxl, myh, myl;
    project_centre(vp, si.mu, p, mxh, mxl, myh, myl);
    Proj P;
    ewa(vp, si, p, P);
    float gmu[3] = {0.f, 0.f, 0.f};

    // opacity
    gr.opacity_logits[i] += g_alpha * P.alpha * (1.f - P.alpha);

    // colour -> SH coefficients and direction
    {
        float dx = si.mu[0] - vp.o[0], dy = si.mu[1] - vp.o[1], dz = si.mu[2] - vp.o[2];
        float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
        float d[3] = {dx * inv, dy * inv, dz * inv};
        float Y[16];
        float3 dY[16];
        sh_eval<DEG>(d[0], d[1], d[2], Y, dY);
        const float* sh = g.sh + i * NSH * 3;
        float* gsh = gr.sh + i * NSH * 3;
        float gd[3] = {0.f, 0.f, 0.f};
        float raw[3], gcol[3];
        sh_colour<NSH, kVecSH>(sh, Y, raw);
        for (int c = 0; c < 3; ++c) gcol[c] = raw[c] > 0.f ? g_rgb[c] : 0.f;   // clamp at 0: no gradient
        if constexpr (kVecSH) {
            const float4* s4 = reinterpret_cast<const float4*>(sh);
            float4* g4 = reinterpret_cast<float4*>(gsh);
#pragma unroll
            for (int q = 0; q < NSH * 3 / 4; ++q) {
                const float4 v = __ldg(s4 + q);
                float4 gv = g4[q];
                const float e[4] = {v.x, v.y, v.z, v.w};
                float* ge[4] = {&gv.x, &gv.y, &gv.z, &gv.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int idx = 4 * q + t, c = idx % 3, k = idx / 3;
                    *ge[t] += gcol[c] * Y[k];
                    const float w = gcol[c] * e[t];
                    gd[0] = fmaf(w, dY[k].x, gd[0]);
                    gd[1] = fmaf(w, dY[k].y, gd[1]);
                    gd[2] = fmaf(w, dY[k].z, gd[2]);
                }
                g4[q] = gv;
            }
        } else {
            for (int c = 0; c < 3; ++c) {
                if (!(raw[c] > 0.f)) continue;
#pragma unroll
                for (int k = 0; k < NSH; ++k) {
                    gsh[3 * k + c] += gcol[c] * Y[k];
                    const float w = gcol[c] * sh[3 * k + c];
                    gd[0] = fmaf(w, dY[k].x, gd[0]);
                    gd[1] = fmaf(w, dY[k].y, gd[1]);
                    gd[2] = fmaf(w, dY[k].z, gd[2]);
                }
            }
        }
        float dd = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
        for (int j = 0; j < 3; ++j) gmu[j] += (gd[j] - d[j] * dd) * inv;
    }

    // conic (a, b, c) = inverse(Sigma'): dL/dSigma' = -Q G Q, G = [[ga, gb/2], [gb/2, gc]]
    float Q00 = P.ca, Q01 = P.cb, Q11 = P.cc;
    float G00 = g_ca, G01 = 0.5f * g_cb, G11 = g_cc;
    float t00 = Q00 * G00 + Q01 * G01, t01 = Q00 * G01 + Q01 * G11;
    float t10 = Q01 * G00 + Q11 * G01, t11 = Q01 * G01 + Q11 * G11;
    float S00 = -(t00 * Q00 + t01 * Q01);
    float S01 = -(t00 * Q01 + t01 * Q11);
    float S11 = -(t10 * Q01 + t11 * Q11);
    // Sigma' = A A^T + dl I:  dL/dA = 2 S A   (S symmetric)
    float GA0[3], GA1[3];
    for (int c = 0; c < 3; ++c) {
        GA0[c] = 2.f * (S00 * P.A0[c] + S01 * P.A1[c]);
        GA1[c] = 2.f * (S01 * P.A0[c] + S11 * P.A1[c]);
    }
    // A[r][c] = s_c (T_r . Rq[:,c]):  dL/ds_c, dL/dRq, dL/dT
    float GT0[3] = {0.f, 0.f, 0.f}, GT1[3] = {0.f, 0.f, 0.f};
    float GRq[9];
    for (int c = 0; c < 3; ++c) {
        float r0 = P.T0[0] * P.Rq[c] + P.T0[1] * P.Rq[3 + c] + P.T0[2] * P.Rq[6 + c];
        float r1 = P.T1[0] * P.Rq[c] + P.T1[1] * P.Rq[3 + c] + P.T1[2] * P.Rq[6 + c];
        float gs = GA0[c] * r0 + GA1[c] * r1;
        gr.log_scales[3 * i + c] += gs * P.s[c];
        float h0 = GA0[c] * P.s[c], h1 = GA1[c] * P.s[c];
        for (int j = 0; j < 3; ++j) {
            GRq[3 * j + c] = h0 * P.T0[j] + h1 * P.T1[j];
            GT0[j] += h0 * P.Rq[3 * j + c];
            GT1[j] += h1 * P.Rq[3 * j + c];
        }
    }
    // T0 = (fx/z)(W0 - u W2), T1 = (fy/z)(W1 - v W2), u = x/z, v = y/z
    float iz = 1.f / P.z;
    float gax = 0.f, gay = 0.f, gu = 0.f, gv = 0.f;
    for (int c = 0; c < 3; ++c) {
        gax += GT0[c] * (vp.R[c] - P.u * vp.R[6 + c]);
        gay += GT1[c] * (vp.R[3 + c] - P.v * vp.R[6 + c]);
        gu -= GT0[c] * vp.fx * iz * vp.R[6 + c];
        gv -= GT1[c] * vp.fy * iz * vp.R[6 + c];
    }
    // mean = (fx u + cx, fy v + cy)
    gu += g_mx * vp.fx;
    gv += g_my * vp.fy;
    // ax = fx/z, ay = fy/z, u = x/z, v = y/z  ->  camera-space centre
    float gp0 = gu * iz;
    float gp1 = gv * iz;
    float gp2 = -(gax * vp.fx + gay * vp.fy) * iz * iz - (gu * P.u + gv * P.v) * iz;
    // p = W mu + t
    for (int j = 0; j < 3; ++j) gmu[j] += vp.R[j] * gp0 + vp.R[3 + j] * gp1 + vp.R[6 + j] * gp2;
    gr.means[3 * i] += gmu[0];
    gr.means[3 * i + 1] += gmu[1];
    gr.means[3 * i + 2] += gmu[2];

    // Rq(w,x,y,z) -> normalised quaternion -> quaternion
    float w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
    float gw = 2.f * (-z * GRq[1] + y * GRq[2] + z * GRq[3] - x * GRq[5] - y * GRq[6] + x * GRq[7]);
    float gx = 2.f * (y * GRq[1] + z * GRq[2] + y * GRq[3] - 2.f * x * GRq[4] - w * GRq[5] + z * GRq[6] + w * GRq[7] -
                      2.f * x * GRq[8]);
    float gy = 2.f * (-2.f * y * GRq[0] + x * GRq[1] + w * GRq[2] + x * GRq[3] + z * GRq[5] - w * GRq[6] + z * GRq[7] -
                      2.f * y * GRq[8]);
    float gz = 2.f * (-2.f * z * GRq[0] - w * GRq[1] + x * GRq[2] + w * GRq[3] - 2.f * z * GRq[4] + y * GRq[5] +
                      x * GRq[6] + y * GRq[7]);
    float dot = gw * w + gx * x + gy * y + gz * z;
    float iq = 1.f / P.qnorm;
    float4* gq = reinterpret_cast<float4*>(gr.quats) + i;
    float4 cur = *gq;
    cur.x += (gw - w * dot) * iq;
    cur.y += (gx - x * dot) * iq;
    cur.z += (gy - y * dot) * iq;
    cur.w += (gz - z * dot) * iq;
    *gq = cur;
}

}  // namespace

// Float4 reads of the SH block need it 16-byte aligned: the base pointer aligned and a
// per-splat stride that is a multiple of 16 bytes (degrees 1 and 3).
static bool vec_sh(const rgs_gaussians& g, const float* gsh = nullptr) {
    const bool stride_ok = g.sh_degree == 1 || g.sh_degree == 3;
    return stride_ok && ((uintptr_t)g.sh % 16 == 0) && (!gsh || (uintptr_t)gsh % 16 == 0);
}

#define RGS_DISPATCH_SH(DEG_EXPR, VEC_EXPR, LAUNCH)                     \
    do {                                                                \
        const bool _vec = (VEC_EXPR);                                   \
        switch (DEG_EXPR) {                                             \
            case 0: { constexpr int D = 0; constexpr bool V = false; LAUNCH; } break; \
            case 1: if (_vec) { constexpr int D = 1; constexpr bool V = true; LAUNCH; } \
                    else { constexpr int D = 1; constexpr bool V = false; LAUNCH; } break; \
            case 2: { constexpr int D = 2; constexpr bool V = false; LAUNCH; } break; \
            default: if (_vec) { constexpr int D = 3; constexpr bool V = true; LAUNCH; } \
                     else { constexpr int D = 3; constexpr bool V = false; LAUNCH; } break; \
        }                                                               \
    } while (0)

namespace {

// ------------------------------------------------------------------ plane templates (Eq. 6)
// Entry i = k L + d of a view's table: the half-plane that level d of leaf k's path puts on
// the image for a splat at depth z, as (z tA) X + (z tB) Y + (z tG + tC) >= 0 with the
// branch's sign folded in (x_i[a] - s = A X + B Y + C along the node's axis a; see
// plane_coeffs), and the clip margin's depth-independent part.
__device__ __forceinline__ void clip_entry(const ViewParams& vp, const TreeParams& tp, int i, float4* plane,
                                           float* margin) {
    const int L = tp.L;
    const int k = i / L, d = i - k * L;
    int node = 0;
    for (int dd = 0; dd < d; ++dd) node = 2 * node + 1 + ((k >> (L - 1 - dd)) & 1);
    const int right = (k >> (L - 1 - d)) & 1;
    const int a = tp.axis[node];
    const float s = tp.split[node];
    const float sg = right ? 1.f : -1.f;
    const float Ra = vp.R[a], Rb = vp.R[3 + a], Rc = vp.R[6 + a];
    const float oa = vp.o[a];
    const float gam = Rc - Ra * vp.cx * vp.ifx - Rb * vp.cy * vp.ify;
    plane[i] = make_float4(sg * Ra * vp.ifx, sg * Rb * vp.ify, sg * gam, sg * (oa - s));
    margin[i] = 1e-5f * (fabsf(oa) + fabsf(s)) + 1e-6f;
}

__global__ void clip_table_kernel(ViewParams vp, TreeParams tp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (1 << tp.L) * tp.L) return;
    clip_entry(vp, tp, i, const_cast<float4*>(vp.clip_plane()), const_cast<float*>(vp.clip_margin()));
}

// One table per request of a batch: blockIdx.y is the slot.
__global__ void clip_table_batch_kernel(const BatchSlot* __restrict__ slots, const BatchHeader* __restrict__ hdr,
                                        TreeParams tp) {
    const int sl = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= hdr->S || i >= (1 << tp.L) * tp.L) return;
    const ViewParams& vp = slots[sl].vp;
    clip_entry(vp, tp, i, const_cast<float4*>(vp.clip_plane()), const_cast<float*>(vp.clip_margin()));
}

}  // namespace

int launch_clip_table(const ViewParams& vp, const TreeParams& tp, cudaStream_t s) {
    const int n = (1 << tp.L) * tp.L;
    if (n == 0) return RGS_OK;
    clip_table_kernel<<<(n + 127) / 128, 128, 0, s>>>(vp, tp);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_clip_table_batch(const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp, cudaStream_t s) {
    const int n = (1 << tp.L) * tp.L;
    if (n == 0) return RGS_OK;
    clip_table_batch_kernel<<<dim3((n + 127) / 128, kMaxSlots), 128, 0, s>>>(slots, hdr, tp);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_project_fwd(const rgs_gaussians& g, const ViewParams& vp, const TreeParams& tp, RasterBuffers& b,
                       cudaStream_t s) {
    unsigned grid = (unsigned)((g.n + 255) / 256);
    if (vp.foot) {
        RGS_DISPATCH_SH(g.sh_degree, vec_sh(g), (project_fwd_kernel<D, V, true><<<grid, 256, 0, s>>>(g, vp, tp, b)));
    } else {
        // the candidate list lives in vis_pos, which the compaction after the projection
        // overwrites; counters[13] counts the candidates (zeroed with the others)
        screen_cull_kernel<<<(unsigned)((g.n + kCullPerBlock - 1) / kCullPerBlock), 256, 0, s>>>(g, vp, b.cnt,
                                                                                               b.vis_pos, b.counters);
        RGS_CUDA_LAUNCH_CHECK();
        RGS_DISPATCH_SH(g.sh_degree, vec_sh(g),
                        (project_cand_kernel<D, V><<<grid, 256, 0, s>>>(g, vp, tp, b, b.vis_pos)));
    }
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_project_batch(const rgs_gaussians& g, const BatchSlot* slots, const BatchHeader* hdr, const TreeParams& tp,
                         const RasterBuffers& b, unsigned long long* counters, cudaStream_t s) {
    const unsigned grid = (unsigned)((g.n + 255) / 256) * (unsigned)kMaxSlots;
    // screen cull first: each slot's candidates to its part of vis_pos (the compaction
    // after the projection overwrites it); the projection then runs on full warps
    const unsigned cgrid = (unsigned)((g.n + kCullPerBlock - 1) / kCullPerBlock) * (unsigned)kMaxSlots;
    screen_cull_batch_kernel<<<cgrid, 256, 0, s>>>(g, slots, hdr, b.cnt, b.vis_pos, counters);
    RGS_CUDA_LAUNCH_CHECK();
    RGS_DISPATCH_SH(g.sh_degree, vec_sh(g),
                    (project_cand_batch_kernel<D, V><<<grid, 256, 0, s>>>(g, slots, hdr, tp, b, counters)));
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

int launch_project_bwd(const rgs_gaussians& g, const rgs_gaussian_grads& gr, const ViewParams& vp,
                       const RasterBuffers& b, cudaStream_t s) {
    unsigned grid = (unsigned)((g.n + 127) / 128);
    RGS_DISPATCH_SH(g.sh_degree, vec_sh(g, gr.sh),
                    (project_bwd_kernel<D, V><<<grid, 128, 0, s>>>(g, gr, vp, b.g2d)));
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

}  // namespace rgs
