// KD partition of Sec. 3.3 on the device.
//
// The tree has depth L and splits level d along axis d mod 3 at the median of the node's
// splat centres, so the K = 2^L leaf boxes hold equal counts (within one) of centres.
// Each axis used is sorted once (stable radix sort of order-preserving float keys); at
// level d a stable one-digit radix pass by node id groups the axis-sorted ids per node
// while keeping them in coordinate order, the medians are read off by position, and every
// splat moves to its child.  The overlapping subsets N_k = {i : the box S_k dilated by D_i
// contains mu_i} are then emitted per splat (ascending leaf) and grouped per leaf with one
// more stable pass, which leaves each list in ascending splat order.
#include <vector>

#include "rgs_internal.cuh"

namespace rgs {
namespace {

__device__ __forceinline__ uint32_t float_key(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void axis_keys_kernel(const float* __restrict__ means, int64_t n, int a, uint32_t* __restrict__ key,
                                 uint32_t* __restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = float_key(means[3 * i + a]);
    val[i] = (uint32_t)i;
}

// key = node index within the level, value = splat id, in the axis-sorted order
__global__ void node_keys_kernel(const uint32_t* __restrict__ axis_sorted, const int32_t* __restrict__ node, int64_t n,
                                 int first, uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t id = axis_sorted[j];
    key[j] = (uint32_t)(node[id] - first);
    val[j] = id;
}

__global__ void node_count_kernel(const int32_t* __restrict__ node, int64_t n, int first, uint32_t* __restrict__ counts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    atomicAdd(&counts[node[i] - first], 1u);
}

// One thread per node of the level: the median split of the node's coordinates, which are
// in ascending order at [start, start + count) of `ordered`.
__global__ void median_kernel(const float* __restrict__ means, const uint32_t* __restrict__ ordered,
                              const uint32_t* __restrict__ counts, int count_nodes, int first, int a,
                              float* __restrict__ split) {
    const int jj = blockIdx.x * blockDim.x + threadIdx.x;
    if (jj >= count_nodes) return;
    uint32_t start = 0;
    for (int q = 0; q < jj; ++q) start += counts[q];
    const uint32_t n = counts[jj];
    float s = 0.f;
    if (n > 0) {
        if (n & 1u) {
            s = means[3 * (size_t)ordered[start + (n - 1) / 2] + a];
        } else {
            float lo = means[3 * (size_t)ordered[start + n / 2 - 1] + a];
            float hi = means[3 * (size_t)ordered[start + n / 2] + a];
            float m = __fadd_rn(__fmul_rn(0.5f, lo), __fmul_rn(0.5f, hi));
            s = (m > lo) ? m : hi;
        }
    }
    split[first + jj] = s;
}

__global__ void descend_kernel(const float* __restrict__ means, int64_t n, int a, const float* __restrict__ split,
                               int32_t* __restrict__ node) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = node[i];
    node[i] = means[3 * i + a] < split[j] ? 2 * j + 1 : 2 * j + 2;
}

// Leaves whose box dilated by D contains mu (left branch mu[a] - D < s, right branch
// mu[a] + D >= s), visited in ascending leaf order.  mode 0 counts, mode 1 writes.
__global__ void subset_pairs_kernel(const float* __restrict__ means, const float* __restrict__ log_scales, int64_t n,
                                    TreeParams tp, float trunc_mult, int mode, uint32_t* __restrict__ cnt,
                                    const uint32_t* __restrict__ off, uint32_t* __restrict__ key,
                                    uint32_t* __restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    float smax = fmaxf(log_scales[3 * i], fmaxf(log_scales[3 * i + 1], log_scales[3 * i + 2]));
    float D = trunc_mult * __expf(smax);
    const int first_leaf = (1 << tp.L) - 1;
    int stack[kMaxKdDepth + 2];
    int sp = 0;
    stack[sp++] = 0;
    uint32_t c = 0;
    uint32_t pos = mode ? off[i] : 0u;
    while (sp > 0) {
        int j = stack[--sp];
        if (j >= first_leaf) {
            if (mode) {
                key[pos + c] = (uint32_t)(j - first_leaf);
                val[pos + c] = (uint32_t)i;
            }
            ++c;
            continue;
        }
        float x = mu[tp.axis[j]];
        float s = tp.split[j];
        if (x + D >= s) stack[sp++] = 2 * j + 2;
        if (x - D < s) stack[sp++] = 2 * j + 1;
    }
    if (!mode) cnt[i] = c;
}

__global__ void leaf_count_kernel(const uint32_t* __restrict__ leaf, int64_t m, uint32_t* __restrict__ counts) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    atomicAdd(&counts[leaf[j]], 1u);
}

unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

struct DevBuf {          // stream-ordered scratch allocations freed on scope exit
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit DevBuf(cudaStream_t st) : s(st) {}
    ~DevBuf() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
    template <typename T>
    T* get(size_t count) {
        void* p = nullptr;
        if (cudaMallocAsync(&p, count * sizeof(T) + 16, s) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return (T*)p;
    }
};

}  // namespace

int kd_build(const rgs_gaussians& g, int L, float trunc_mult, KdBuild* out, cudaStream_t s) {
    const int64_t N = g.n;
    const int K = 1 << L;
    out->L = L;
    out->idx_dev = nullptr;
    out->M = 0;
    for (int j = 0; j < kMaxNodes; ++j) {
        out->axis[j] = 0;
        out->split[j] = 0.f;
    }
    DevBuf buf(s);
    uint32_t* ka = buf.get<uint32_t>(N);
    uint32_t* va = buf.get<uint32_t>(N);
    uint32_t* kb = buf.get<uint32_t>(N);
    uint32_t* vb = buf.get<uint32_t>(N);
    int32_t* node = buf.get<int32_t>(N);
    uint32_t* cnt = buf.get<uint32_t>(N);
    uint32_t* off = buf.get<uint32_t>(N);
    float* split_dev = buf.get<float>(kMaxNodes + 1);
    uint32_t* node_counts = buf.get<uint32_t>(K + 1);
    size_t tbytes = radix_temp_bytes(N) + scan_temp_bytes(N);
    void* temp = buf.get<char>(tbytes);
    if (!ka || !va || !kb || !vb || !node || !cnt || !off || !split_dev || !node_counts || !temp) {
        set_error("kd_partition: device allocation failed");
        return RGS_ENOMEM;
    }
    const int naxes = L < 3 ? L : 3;
    uint32_t* axis_sorted[3] = {nullptr, nullptr, nullptr};
    for (int a = 0; a < naxes; ++a) {
        axis_sorted[a] = buf.get<uint32_t>(N);
        if (!axis_sorted[a]) {
            set_error("kd_partition: device allocation failed");
            return RGS_ENOMEM;
        }
        axis_keys_kernel<<<blocks(N), 256, 0, s>>>(g.means, N, a, ka, va);
        RGS_CUDA_LAUNCH_CHECK();
        bool alt = false;
        int rc = radix_sort_pairs(ka, va, kb, vb, N, 32, temp, tbytes, s, &alt);
        if (rc) return rc;
        RGS_CUDA_TRY(cudaMemcpyAsync(axis_sorted[a], alt ? vb : va, sizeof(uint32_t) * N, cudaMemcpyDeviceToDevice, s));
    }
    RGS_CUDA_TRY(cudaMemsetAsync(node, 0, sizeof(int32_t) * N, s));
    RGS_CUDA_TRY(cudaMemsetAsync(split_dev, 0, sizeof(float) * kMaxNodes, s));
    for (int d = 0; d < L; ++d) {
        const int a = d % 3;
        const int first = (1 << d) - 1, count_nodes = 1 << d;
        const uint32_t* ordered = axis_sorted[a];
        if (d > 0) {
            node_keys_kernel<<<blocks(N), 256, 0, s>>>(axis_sorted[a], node, N, first, ka, va);
            RGS_CUDA_LAUNCH_CHECK();
            bool alt = false;
            int rc = radix_sort_pairs(ka, va, kb, vb, N, d, temp, tbytes, s, &alt);
            if (rc) return rc;
            ordered = alt ? vb : va;
        }
        RGS_CUDA_TRY(cudaMemsetAsync(node_counts, 0, sizeof(uint32_t) * count_nodes, s));
        node_count_kernel<<<blocks(N), 256, 0, s>>>(node, N, first, node_counts);
        RGS_CUDA_LAUNCH_CHECK();
        median_kernel<<<blocks(count_nodes, 64), 64, 0, s>>>(g.means, ordered, node_counts, count_nodes, first, a,
                                                            split_dev);
        RGS_CUDA_LAUNCH_CHECK();
        descend_kernel<<<blocks(N), 256, 0, s>>>(g.means, N, a, split_dev, node);
        RGS_CUDA_LAUNCH_CHECK();
        out->axis[first] = (int8_t)a;
        for (int jj = 0; jj < count_nodes; ++jj) out->axis[first + jj] = (int8_t)a;
    }
    if (K > 1) RGS_CUDA_TRY(cudaMemcpyAsync(out->split, split_dev, sizeof(float) * (K - 1), cudaMemcpyDeviceToHost, s));
    RGS_CUDA_TRY(cudaStreamSynchronize(s));
    return kd_subsets(g, trunc_mult, out, s);
}

int kd_subsets(const rgs_gaussians& g, float trunc_mult, KdBuild* out, cudaStream_t s) {
    const int64_t N = g.n;
    const int L = out->L;
    const int K = 1 << L;
    DevBuf buf(s);
    uint32_t* cnt = buf.get<uint32_t>(N);
    uint32_t* off = buf.get<uint32_t>(N);
    uint32_t* node_counts = buf.get<uint32_t>(K + 1);
    size_t tbytes = scan_temp_bytes(N);
    void* temp = buf.get<char>(tbytes);
    if (!cnt || !off || !node_counts || !temp) {
        set_error("kd_partition: device allocation failed");
        return RGS_ENOMEM;
    }
    // subsets N_k
    TreeParams tp;
    tp.L = L;
    for (int j = 0; j < kMaxNodes; ++j) {
        tp.axis[j] = out->axis[j];
        tp.split[j] = out->split[j];
    }
    subset_pairs_kernel<<<blocks(N), 256, 0, s>>>(g.means, g.log_scales, N, tp, trunc_mult, 0, cnt, nullptr, nullptr,
                                                  nullptr);
    RGS_CUDA_LAUNCH_CHECK();
    int rc = exclusive_scan_u32(cnt, off, N, 0, nullptr, temp, tbytes, s);
    if (rc) return rc;
    uint32_t last_off = 0, last_cnt = 0;
    RGS_CUDA_TRY(cudaMemcpyAsync(&last_off, off + (N - 1), 4, cudaMemcpyDeviceToHost, s));
    RGS_CUDA_TRY(cudaMemcpyAsync(&last_cnt, cnt + (N - 1), 4, cudaMemcpyDeviceToHost, s));
    RGS_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t M = (int64_t)last_off + last_cnt;
    uint32_t* pk = buf.get<uint32_t>(M);
    uint32_t* pv = buf.get<uint32_t>(M);
    uint32_t* pk2 = buf.get<uint32_t>(M);
    uint32_t* pv2 = buf.get<uint32_t>(M);
    size_t t2 = radix_temp_bytes(M);
    void* temp2 = buf.get<char>(t2);
    if (!pk || !pv || !pk2 || !pv2 || !temp2) {
        set_error("kd_partition: device allocation failed");
        return RGS_ENOMEM;
    }
    subset_pairs_kernel<<<blocks(N), 256, 0, s>>>(g.means, g.log_scales, N, tp, trunc_mult, 1, nullptr, off, pk, pv);
    RGS_CUDA_LAUNCH_CHECK();
    bool alt = false;
    rc = radix_sort_pairs(pk, pv, pk2, pv2, M, L, temp2, t2, s, &alt);
    if (rc) return rc;
    RGS_CUDA_TRY(cudaMemsetAsync(node_counts, 0, sizeof(uint32_t) * K, s));
    leaf_count_kernel<<<blocks(M), 256, 0, s>>>(alt ? pk2 : pk, M, node_counts);
    RGS_CUDA_LAUNCH_CHECK();
    std::vector<uint32_t> lc(K);
    RGS_CUDA_TRY(cudaMemcpyAsync(lc.data(), node_counts, sizeof(uint32_t) * K, cudaMemcpyDeviceToHost, s));
    int32_t* idx = nullptr;
    RGS_CUDA_TRY(cudaMalloc(&idx, sizeof(int32_t) * (M > 0 ? M : 1)));
    cudaError_t e = cudaMemcpyAsync(idx, alt ? pv2 : pv, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(idx);
        set_error("kd_partition: %s", cudaGetErrorString(e));
        return RGS_ECUDA;
    }
    out->offsets[0] = 0;
    for (int k = 0; k < K; ++k) out->offsets[k + 1] = out->offsets[k] + lc[k];
    out->idx_dev = idx;
    out->M = M;
    return RGS_OK;
}

}  // namespace rgs
