// lidar.cu -- LiDAR elevation supervision (RoGs Sec. 3.3.2, L_z).
//
// Targets (once per point cloud): zbar_i = z of the LiDAR point nearest to
// surfel i in the xy-plane, among points within radius r (NaN if none; ties
// to the lower point index).  The points are bucketed by a spatial hash of
// their xy cell (cell side slightly above r, so a point within r of a surfel
// lies in the 3 x 3 cells around the surfel's cell), sorted by bucket with the
// library's radix sort, and each surfel scans the buckets of those 9 cells;
// a point that only shares a bucket by hash collision fails the distance test.
//
// Loss (every step): L_z = sum_i (z_i - zbar_i)^2 over surfels with a target,
// dL/dz_i = 2 (z_i - zbar_i); loss[0] += lambda_z L_z, summed in a fixed order.
#include "kernels.h"

namespace rogs {

__device__ __forceinline__ uint32_t cell_bucket(int cx, int cy, uint32_t mask) {
    return ((uint32_t)cx * 73856093u ^ (uint32_t)cy * 19349663u) & mask;
}

__global__ void __launch_bounds__(256) lidar_hash_k(const float* __restrict__ pts, long long m, float inv_cell,
                                                    uint32_t mask, uint32_t* __restrict__ keys,
                                                    uint32_t* __restrict__ vals) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < m; i += (long long)gridDim.x * 256) {
        const int cx = (int)floorf(pts[3 * i] * inv_cell), cy = (int)floorf(pts[3 * i + 1] * inv_cell);
        keys[i] = cell_bucket(cx, cy, mask);
        vals[i] = (uint32_t)i;
    }
}

// Bucket [start, end) of the sorted keys and the points in sorted order
// (x, y, z, original index) for the queries.
__global__ void __launch_bounds__(256) lidar_ranges_k(const uint32_t* __restrict__ keys,
                                                      const uint32_t* __restrict__ order,
                                                      const float* __restrict__ pts, long long m,
                                                      uint2* __restrict__ ranges, float4* __restrict__ sorted) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    for (long long p = blockIdx.x * 256ll + threadIdx.x; p < m; p += (long long)gridDim.x * 256) {
        const uint32_t b = keys[p];
        if (p == 0 || keys[p - 1] != b) ranges[b].x = (uint32_t)p;
        if (p + 1 == m || keys[p + 1] != b) ranges[b].y = (uint32_t)(p + 1);
        const uint32_t i = order[p];
        sorted[p] = make_float4(pts[3ull * i], pts[3ull * i + 1], pts[3ull * i + 2], __uint_as_float(i));
    }
}

__global__ void __launch_bounds__(256) lidar_nearest_k(const float* __restrict__ xyz, long long n,
                                                       const float4* __restrict__ sorted,
                                                       const uint2* __restrict__ ranges, uint32_t mask,
                                                       float inv_cell, float r2, float* __restrict__ zbar) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const float x = xyz[3 * i], y = xyz[3 * i + 1];
        const int cx = (int)floorf(x * inv_cell), cy = (int)floorf(y * inv_cell);
        float best = 3.0e38f, bz = __int_as_float(0x7fc00000);   // NaN: no point within r
        uint32_t bi = 0xffffffffu;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const uint2 rg = ranges[cell_bucket(cx + dx, cy + dy, mask)];
                for (uint32_t p = rg.x; p < rg.y; ++p) {
                    const float4 q = sorted[p];
                    const float ex = q.x - x, ey = q.y - y;
                    const float d2 = fmaf(ex, ex, ey * ey);
                    const uint32_t qi = __float_as_uint(q.w);
                    if (d2 <= r2 && (d2 < best || (d2 == best && qi < bi))) {
                        best = d2;
                        bi = qi;
                        bz = q.z;
                    }
                }
            }
        zbar[i] = bz;
    }
}

__global__ void __launch_bounds__(256) elev_k(const float* __restrict__ xyz, long long n,
                                              const float* __restrict__ zbar, float lambda,
                                              float* __restrict__ grad_xyz, float* __restrict__ partials) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ float sh[8];
    float acc = 0.0f;
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const float t = zbar[i];
        if (!(t == t)) continue;   // no target
        const float d = xyz[3 * i + 2] - t;
        acc = fmaf(d, d, acc);
        if (grad_xyz) grad_xyz[3 * i + 2] += 2.0f * lambda * d;   // one thread per surfel: no race
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < 8; ++w) t += sh[w];
        partials[blockIdx.x] = t;
    }
}

__global__ void elev_final_k(const float* __restrict__ partials, int n, float lambda, float* __restrict__ loss) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    float s = 0.0f;
    for (int i = threadIdx.x; i < n; i += 32) s += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (threadIdx.x == 0) loss[0] += lambda * s;
}

int elev_blocks() { return 152 * 8; }

static int grid_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

int lidar_bucket_bits(long long m) {
    int b = 10;
    while (b < 26 && (1ll << b) < 2 * m) ++b;
    return b;
}

void lidar_targets(const float* xyz, long long n, const float* pts, long long m, float radius, LidarScratch& w,
                   float* zbar, cudaStream_t s) {
    const int bits = lidar_bucket_bits(m);
    const uint32_t mask = (1u << bits) - 1u;
    const float cell = radius * 1.001f + 1e-6f;   // a point within r is at most one cell away
    const float inv_cell = 1.0f / cell;
    cudaMemsetAsync(w.ranges, 0, sizeof(uint2) << bits, s);
    if (m > 0) {
        launch_pdl(lidar_hash_k, dim3(grid_for(m)), dim3(256), 0, s, pts, m, inv_cell, mask, w.keys, w.vals);
        radix_sort_pairs(w.keys, w.vals, w.skeys, w.svals, w.kalt, w.valt, nullptr, (unsigned long long)m, bits,
                         w.hist, s, 2048);
        launch_pdl(lidar_ranges_k, dim3(grid_for(m)), dim3(256), 0, s, w.skeys, w.svals, pts, m, w.ranges, w.sorted);
        note_launches(2);
    }
    if (n > 0) {
        launch_pdl(lidar_nearest_k, dim3(grid_for(n)), dim3(256), 0, s, xyz, n, w.sorted, w.ranges, mask, inv_cell, radius * radius,
                                                     zbar);
        note_launches(1);
    }
}

void elev_loss(const float* xyz, long long n, const float* zbar, float lambda, float* loss, float* grad_xyz,
               float* partials, cudaStream_t s) {
    long long nb = (n + 255) / 256;
    if (nb > elev_blocks()) nb = elev_blocks();
    if (nb < 1) nb = 1;
    launch_pdl(elev_k, dim3((int)nb), dim3(256), 0, s, xyz, n, zbar, lambda, grad_xyz, partials);
    launch_pdl(elev_final_k, dim3(1), dim3(32), 0, s, partials, (int)nb, lambda, loss);
    note_launches(2);
}

}  // namespace rogs
