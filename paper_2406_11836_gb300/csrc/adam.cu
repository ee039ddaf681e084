// Fused Adam step over a flat parameter buffer (Sec. 4 implementation details: the
// position learning rate decays exponentially; every parameter group has its own rate).
// One pass reads p, g, m, v and writes p, m, v (and optionally zeroes the non-zero parts
// of g) with 16-byte vector accesses: 28 (up to 32) bytes per parameter, so the kernel is
// bound by HBM bandwidth.
#include "rgs_internal.cuh"

namespace rgs {
namespace {

struct AdamSegs {
    int64_t off[17];
    float lr[16];
    int nseg;
    // optional periodic rule inside segment pseg (-1: none): an element whose offset from
    // the segment start is below `head` modulo `period` takes head_lr (the degree-0 SH
    // coefficients of every splat in a [N, (d+1)^2, 3] block)
    int pseg;
    int64_t period, head;
    float head_lr;
};

__device__ __forceinline__ int seg_of(const AdamSegs& s, int64_t i) {
    int q = 0;
    while (q + 1 < s.nseg && i >= s.off[q + 1]) ++q;
    return q;
}

__device__ __forceinline__ float seg_lr(const AdamSegs& s, int64_t i) { return s.lr[seg_of(s, i)]; }

// Rate of element i whose position in the period is pos (valid when segment pseg holds i).
__device__ __forceinline__ float elem_lr(const AdamSegs& s, int64_t i, int64_t pos) {
    const int q = seg_of(s, i);
    return (q == s.pseg && pos < s.head) ? s.head_lr : s.lr[q];
}

__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, float lr, float b1, float b2, float eps,
                                      float bc1, float bc2) {
    m = fmaf(b1, m, (1.f - b1) * g);
    v = fmaf(b2, v, (1.f - b2) * g * g);
    p -= lr * (m * bc1) / (sqrtf(v * bc2) + eps);
}

__global__ void __launch_bounds__(256)
adam_kernel(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v, int64_t n,
            AdamSegs segs, float b1, float b2, float eps, float bc1, float bc2, int zero_grad) {
    const int64_t n4 = n / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float4* p4 = reinterpret_cast<float4*>(p);
    float4* g4 = reinterpret_cast<float4*>(g);
    float4* m4 = reinterpret_cast<float4*>(m);
    float4* v4 = reinterpret_cast<float4*>(v);
    // position of element 4 i in the period of the periodic segment, carried along the
    // grid-stride loop (one 64-bit remainder per thread, then additions)
    const int64_t i_first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool periodic = segs.pseg >= 0;
    const int64_t per = periodic ? segs.period : 1;
    const int64_t step_mod = (4 * stride) % per;
    int64_t r = (((4 * i_first - (periodic ? segs.off[segs.pseg] : 0)) % per) + per) % per;
    for (int64_t i = i_first; i < n4; i += stride) {
        float4 P = p4[i], G = g4[i], M = m4[i], V = v4[i];
        const int64_t e = 4 * i;
        float l0, l1, l2, l3;
        if (periodic) {
            const int q0 = seg_of(segs, e), q3 = seg_of(segs, e + 3);
            if (q0 == q3) {   // four elements of one segment
                const float lq = segs.lr[q0];
                if (q0 != segs.pseg) {
                    l0 = l1 = l2 = l3 = lq;
                } else {
                    const int64_t r1 = r + 1 >= per ? r + 1 - per : r + 1, r2 = r1 + 1 >= per ? r1 + 1 - per : r1 + 1,
                                  r3 = r2 + 1 >= per ? r2 + 1 - per : r2 + 1;
                    l0 = r < segs.head ? segs.head_lr : lq;
                    l1 = r1 < segs.head ? segs.head_lr : lq;
                    l2 = r2 < segs.head ? segs.head_lr : lq;
                    l3 = r3 < segs.head ? segs.head_lr : lq;
                }
            } else {
                const int64_t r1 = r + 1 >= per ? r + 1 - per : r + 1, r2 = r1 + 1 >= per ? r1 + 1 - per : r1 + 1,
                              r3 = r2 + 1 >= per ? r2 + 1 - per : r2 + 1;
                l0 = elem_lr(segs, e, r);
                l1 = elem_lr(segs, e + 1, r1);
                l2 = elem_lr(segs, e + 2, r2);
                l3 = elem_lr(segs, e + 3, r3);
            }
            r += step_mod;
            if (r >= per) r -= per;
        } else {
            l0 = seg_lr(segs, e);
            l3 = seg_lr(segs, e + 3);
            l1 = l0 == l3 ? l0 : seg_lr(segs, e + 1);
            l2 = l0 == l3 ? l0 : seg_lr(segs, e + 2);
        }
        adam1(P.x, G.x, M.x, V.x, l0, b1, b2, eps, bc1, bc2);
        adam1(P.y, G.y, M.y, V.y, l1, b1, b2, eps, bc1, bc2);
        adam1(P.z, G.z, M.z, V.z, l2, b1, b2, eps, bc1, bc2);
        adam1(P.w, G.w, M.w, V.w, l3, b1, b2, eps, bc1, bc2);
        p4[i] = P;
        m4[i] = M;
        v4[i] = V;
        // most splats of a view get no gradient: skip storing zeros over zeros
        if (zero_grad && (G.x != 0.f || G.y != 0.f || G.z != 0.f || G.w != 0.f))
            g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // scalar tail
    const int64_t t = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        float P = p[t], M = m[t], V = v[t];
        const float lt = periodic ? elem_lr(segs, t, (((t - segs.off[segs.pseg]) % per) + per) % per)
                                  : seg_lr(segs, t);
        adam1(P, g[t], M, V, lt, b1, b2, eps, bc1, bc2);
        p[t] = P;
        m[t] = M;
        v[t] = V;
        if (zero_grad) g[t] = 0.f;
    }
}

}  // namespace

int launch_adam(float* p, float* g, float* m, float* v, int64_t n, const int64_t* seg_off, const float* seg_lr_h,
                int nseg, float b1, float b2, float eps, float bc1, float bc2, int zero_grad, cudaStream_t s,
                int pseg, int64_t period, int64_t head, float head_lr) {
    AdamSegs segs;
    segs.nseg = nseg;
    segs.pseg = pseg;
    segs.period = period;
    segs.head = head;
    segs.head_lr = head_lr;
    for (int q = 0; q <= nseg; ++q) segs.off[q] = seg_off[q];
    for (int q = 0; q < nseg; ++q) segs.lr[q] = seg_lr_h[q];
    const int sms = sm_count();
    int64_t want = (n / 4 + 255) / 256;
    int64_t cap = (int64_t)sms * 8;
    unsigned grid = (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
    adam_kernel<<<grid, 256, 0, s>>>(p, g, m, v, n, segs, b1, b2, eps, bc1, bc2, zero_grad);
    RGS_CUDA_LAUNCH_CHECK();
    return RGS_OK;
}

}  // namespace rgs
