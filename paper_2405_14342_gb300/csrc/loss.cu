// loss.cu -- masked L1 colour and masked cross-entropy semantic loss
// (RoGs Sec. 3.3.2, Eqs. 8 and 9, weighted as in Eq. 12) and its gradient
// with respect to the rendered planes.
//
//   mask_count_k : |M| = number of mask pixels over all views
//   loss_k       : per pixel, L1 over the three colour channels and the
//                  log-softmax cross entropy of the C logits; writes dL/dout
//                  (one thread per pixel, coalesced plane reads/writes) and a
//                  per-block partial sum
//   loss_final_k : deterministic sum of the partials (fixed order), / |M|
#include "kernels.h"

namespace rogs {

constexpr int kLossThreads = 256;

int loss_blocks(long long total_pixels) { return (int)((total_pixels + kLossThreads - 1) / kLossThreads); }

__device__ __forceinline__ int view_of_pixel(const ViewParams* views, int n_views, long long p) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (views[mid].pix_base <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kLossThreads) mask_count_k(const uint8_t* __restrict__ mask, long long n,
                                                             unsigned long long* __restrict__ counter) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ unsigned int sh[kLossThreads / 32];
    unsigned int c = 0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        c += mask[p] ? 1u : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kLossThreads / 32; ++w) t += sh[w];
        if (t) atomicAdd(counter, t);
    }
}

__global__ void __launch_bounds__(kLossThreads) loss_k(const ViewParams* __restrict__ views, int n_views,
                                                       long long total_pixels, int C, const float* __restrict__ out,
                                                       const Targets tg, float lambda_c,
                                                       float lambda_s, const unsigned long long* __restrict__ counter,
                                                       float* __restrict__ grad_out, float* __restrict__ partials) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ float sh[kLossThreads / 32];
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (p < total_pixels) {
        const int vi = view_of_pixel(views, n_views, p);
        const ViewParams& v = views[vi];
        const long long q = p - v.pix_base;
        const long long plane = (long long)v.W * v.H;
        const int nch = 3 + C + 1;
        const float* o = out + (long long)nch * v.pix_base + q;
        float* g = grad_out + (long long)nch * v.pix_base + q;
        const unsigned long long nm = *counter;
        const bool m = tg.mask[p] != 0 && nm > 0;
        if (!m) {
            for (int ch = 0; ch < nch; ++ch) g[ch * plane] = 0.0f;
        } else {
            const float inv = 1.0f / (float)nm;
            float tr[3];
            int lb;
            load_pixel_target(tg, 3ll * v.pix_base + q, plane, p, C, tr[0], tr[1], tr[2], lb);
            float l1 = 0.0f;
            for (int ch = 0; ch < 3; ++ch) {
                const float d = o[ch * plane] - tr[ch];
                l1 += fabsf(d);
                g[ch * plane] = lambda_c * inv * (d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f));
            }
            float ce = 0.0f;
            if (lb >= 0 && lb < C) {  // labels outside [0, C) carry no semantic term
                // softmax with one exponential per class: e = exp(x - max), p = e / sum e
                float mx = o[3 * plane];
                for (int ch = 1; ch < C; ++ch) mx = fmaxf(mx, o[(3 + ch) * plane]);
                float se = 0.0f;
                for (int ch = 0; ch < C; ++ch) se += __expf(o[(3 + ch) * plane] - mx);
                ce = mx + logf(se) - o[(3 + lb) * plane];
                const float rse = 1.0f / se;
                const float ls = lambda_s * inv;
                for (int ch = 0; ch < C; ++ch) {
                    const float e = __expf(o[(3 + ch) * plane] - mx);
                    g[(3 + ch) * plane] = ls * (e * rse - (ch == lb ? 1.0f : 0.0f));
                }
            } else {
                for (int ch = 0; ch < C; ++ch) g[(3 + ch) * plane] = 0.0f;
            }
            g[(3 + C) * plane] = 0.0f;
            l = lambda_c * l1 + lambda_s * ce;
        }
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) l += __shfl_xor_sync(kFull, l, o2);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < kLossThreads / 32; ++w) t += sh[w];
        partials[blockIdx.x] = t;
    }
}

// FP64 is slow on this part, so the partials are summed in FP32: each of
// 1024 threads adds its strided share (loads unrolled so they overlap), then
// a fixed-order tree; the result does not depend on timing.
__global__ void __launch_bounds__(1024) loss_final_k(const float* __restrict__ partials, int n,
                                                     const unsigned long long* __restrict__ counter,
                                                     const float* __restrict__ extra, float* __restrict__ loss) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ float sh[32];
    // thread t sums the float4 groups t, t + 1024, ... (all loads in flight at
    // once, eight independent accumulators) and the tail; the order is fixed
    float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int n4 = n / 4;
    const float4* p4 = reinterpret_cast<const float4*>(partials);
    int i = threadIdx.x;
    for (; i + 1024 < n4; i += 2048) {
        const float4 x = p4[i], y = p4[i + 1024];
        a[0] += x.x; a[1] += x.y; a[2] += x.z; a[3] += x.w;
        a[4] += y.x; a[5] += y.y; a[6] += y.z; a[7] += y.w;
    }
    if (i < n4) {
        const float4 x = p4[i];
        a[0] += x.x; a[1] += x.y; a[2] += x.z; a[3] += x.w;
    }
    if (threadIdx.x < n - 4 * n4) a[0] += partials[4 * n4 + threadIdx.x];
    float s = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = sh[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
        if (threadIdx.x == 0) {
            const unsigned long long nm = *counter;
            loss[0] = (nm ? t / (float)nm : 0.0f) + (extra ? extra[0] : 0.0f);
        }
    }
}

void loss_fwd_bwd(const ViewParams* views, int n_views, long long total_pixels, int C, const float* out,
                  const Targets& tg, float lambda_c, float lambda_s,
                  float* loss, float* grad_out, unsigned long long* counter, float* partials, int n_blocks_cap,
                  cudaStream_t s) {
    const int nb = loss_blocks(total_pixels);
    cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    int gc = nb < 152 * 8 ? nb : 152 * 8;
    if (gc < 1) gc = 1;
    launch_pdl(mask_count_k, dim3(gc), dim3(kLossThreads), 0, s, tg.mask, total_pixels, counter);
    launch_pdl(loss_k, dim3(nb > 0 ? nb : 1), dim3(kLossThreads), 0, s, views, n_views, total_pixels, C, out, tg,
               lambda_c, lambda_s, counter, grad_out, partials);
    launch_pdl(loss_final_k, dim3(1), dim3(1024), 0, s, partials, nb, counter, nullptr, loss);
    note_launches(3);
    (void)n_blocks_cap;
}

void mask_count(const uint8_t* mask, long long total_pixels, unsigned long long* counter, cudaStream_t s) {
    cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    long long nb = (total_pixels + kLossThreads - 1) / kLossThreads;
    int gc = (int)(nb < 152 * 8 ? nb : 152 * 8);
    if (gc < 1) gc = 1;
    launch_pdl(mask_count_k, dim3(gc), dim3(kLossThreads), 0, s, mask, total_pixels, counter);
    note_launches(1);
}

void loss_final(const float* partials, int n, const unsigned long long* counter, const float* extra, float* loss,
                cudaStream_t s) {
    launch_pdl(loss_final_k, dim3(1), dim3(1024), 0, s, partials, n, counter, extra, loss);
    note_launches(1);
}

}  // namespace rogs
