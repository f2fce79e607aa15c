// smooth.cu -- elevation smoothness loss over the grid index map.
//
// RoGs Sec. 3.3.2 (smoothness loss) with the neighbour lookup of the
// supplementary "Smooth Loss K Nearest Neighbor Acceleration": the K = 4
// neighbours of a surfel are the surfels at the grid vertices above, below,
// left and right of its own vertex; a vertex off the grid or off the road
// (-1) stands for the surfel itself.
//
//   L = (1/4) sum_i sum_{j in N(i)} (z_i - z_j)^2
//   dL/dz_i = sum over the vertex pairs (v_i, v_j) adjacent in the grid of
//             (z_i - z_j)   (each ordered pair contributes 2 (z_i - z_j) / 4
//             to z_i from i's sum and the same from j's sum)
//
// One thread per grid vertex (a stencil over the index map, grid-stride over
// a fixed persistent grid); the loss leaves as one partial per CTA, summed in
// a fixed order by a single-block kernel, so it does not depend on timing.
#include "kernels.h"

namespace rogs {

constexpr int kSmoothThreads = 256;

__global__ void __launch_bounds__(kSmoothThreads) smooth_k(const int32_t* __restrict__ gi, int W, int H,
                                                            const float* __restrict__ xyz, float lambda,
                                                            float* __restrict__ grad_xyz,
                                                            float* __restrict__ partials) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ float sh[kSmoothThreads / 32];
    const long long cells = (long long)W * H;
    float acc = 0.0f;
    for (long long cell = blockIdx.x * (long long)kSmoothThreads + threadIdx.x; cell < cells;
         cell += (long long)gridDim.x * kSmoothThreads) {
        const int i = gi[cell];
        if (i < 0) continue;
        const int r = (int)(cell / W), c = (int)(cell - (long long)r * W);
        const int nb[4] = {r > 0 ? gi[cell - W] : -1, r + 1 < H ? gi[cell + W] : -1, c > 0 ? gi[cell - 1] : -1,
                           c + 1 < W ? gi[cell + 1] : -1};
        const float zi = xyz[3ll * i + 2];
        float l = 0.0f, g = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = nb[k] >= 0 ? nb[k] : i;
            const float d = zi - xyz[3ll * j + 2];
            l = fmaf(d, d, l);
            g += d;
        }
        acc += l;
        if (grad_xyz && g != 0.0f) atomicAdd(&grad_xyz[3ll * i + 2], lambda * g);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < kSmoothThreads / 32; ++w) t += sh[w];
        partials[blockIdx.x] = t;
    }
}

// loss[0] = lambda / 4 * (sum of the partials), 32 lanes in a fixed order.
__global__ void smooth_final_k(const float* __restrict__ partials, int n, float lambda, float* __restrict__ loss) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    float s = 0.0f;
    for (int i = threadIdx.x; i < n; i += 32) s += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (threadIdx.x == 0) loss[0] = 0.25f * lambda * s;
}

int smooth_blocks() { return 152 * 8; }

void smooth_loss(const int32_t* grid_index, int grid_w, int grid_h, const float* xyz, float lambda, float* loss,
                 float* grad_xyz, float* partials, cudaStream_t s) {
    const long long cells = (long long)grid_w * grid_h;
    long long nb = (cells + kSmoothThreads - 1) / kSmoothThreads;
    if (nb > smooth_blocks()) nb = smooth_blocks();
    if (nb < 1) nb = 1;
    launch_pdl(smooth_k, dim3((int)nb), dim3(kSmoothThreads), 0, s, grid_index, grid_w, grid_h, xyz, lambda, grad_xyz, partials);
    launch_pdl(smooth_final_k, dim3(1), dim3(32), 0, s, partials, (int)nb, lambda, loss);
    note_launches(2);
}

}  // namespace rogs
