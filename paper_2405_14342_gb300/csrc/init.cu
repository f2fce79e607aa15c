// init.cu -- pose-based initialisation of surfel height and rotation
// (RoGs Sec. 3.2, Eq. 4; supplementary "Height Initialization", Eqs. S1-S2).
//
// For every grid point (x_i, y_i): the nearest vehicle pose in the xy plane
// (binary32 squared distance (dx*dx)+(dy*dy), ties to the lowest index),
// then the height that puts the surfel in the pose's xy plane,
//   n3 . (x_i - x_v, y_i - y_v, z_i - z_v) = 0,  n3 = third column of R_v,
// or z_i = z_v under the small-roll reading; the rotation is R_v, stored as a
// unit quaternion (w, x, y, z) with w >= 0.  Poses are staged through shared
// memory in chunks; one thread per surfel.
#include "kernels.h"

namespace rogs {

constexpr int kInitThreads = 256;
constexpr int kPoseChunk = 512;

__device__ __forceinline__ float4 quat_from_rotation(const float* R) {
    // Shepperd's method on the largest of trace and diagonal entries
    const float r00 = R[0], r01 = R[1], r02 = R[2], r10 = R[3], r11 = R[4], r12 = R[5], r20 = R[6], r21 = R[7],
                r22 = R[8];
    const float tr = r00 + r11 + r22;
    float w, x, y, z;
    if (tr > 0.0f) {
        const float s = sqrtf(tr + 1.0f) * 2.0f;
        w = 0.25f * s; x = (r21 - r12) / s; y = (r02 - r20) / s; z = (r10 - r01) / s;
    } else if (r00 > r11 && r00 > r22) {
        const float s = sqrtf(1.0f + r00 - r11 - r22) * 2.0f;
        w = (r21 - r12) / s; x = 0.25f * s; y = (r01 + r10) / s; z = (r02 + r20) / s;
    } else if (r11 > r22) {
        const float s = sqrtf(1.0f + r11 - r00 - r22) * 2.0f;
        w = (r02 - r20) / s; x = (r01 + r10) / s; y = 0.25f * s; z = (r12 + r21) / s;
    } else {
        const float s = sqrtf(1.0f + r22 - r00 - r11) * 2.0f;
        w = (r10 - r01) / s; x = (r02 + r20) / s; y = (r12 + r21) / s; z = 0.25f * s;
    }
    const float n = rsqrtf(w * w + x * x + y * y + z * z);
    const float sg = w < 0.0f ? -n : n;
    return make_float4(w * sg, x * sg, y * sg, z * sg);
}

__global__ void __launch_bounds__(kInitThreads) init_k(const float* __restrict__ grid_xy, long long n,
                                                       const float* __restrict__ poses, long long n_poses,
                                                       int exact_plane, float* __restrict__ out_z,
                                                       float* __restrict__ out_quat,
                                                       int32_t* __restrict__ out_nearest) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    __shared__ float2 sp[kPoseChunk];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float x = 0.0f, y = 0.0f;
    if (i < n) {
        const float2 g = reinterpret_cast<const float2*>(grid_xy)[i];
        x = g.x;
        y = g.y;
    }
    long long best = -1;
    float bd = 0.0f;
    for (long long c0 = 0; c0 < n_poses; c0 += kPoseChunk) {
        const int m = (int)min((long long)kPoseChunk, n_poses - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += blockDim.x)
            sp[t] = make_float2(poses[12 * (c0 + t)], poses[12 * (c0 + t) + 1]);
        __syncthreads();
        for (int t = 0; t < m; ++t) {
            const float dx = __fsub_rn(x, sp[t].x);
            const float dy = __fsub_rn(y, sp[t].y);
            const float d = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            if (best < 0 || d < bd) {
                bd = d;
                best = c0 + t;
            }
        }
    }
    if (i >= n || best < 0) return;
    const float* pv = poses + 12 * best;
    const float* R = pv + 3;
    float z = pv[2];
    if (exact_plane) {
        const float n31 = R[2], n32 = R[5], n33 = R[8];
        z = pv[2] - (n31 * (x - pv[0]) + n32 * (y - pv[1])) / n33;
    }
    out_z[i] = z;
    reinterpret_cast<float4*>(out_quat)[i] = quat_from_rotation(R);
    if (out_nearest) out_nearest[i] = (int32_t)best;
}

void init_from_poses(const float* grid_xy, long long n, const float* poses_dev, long long n_poses, int exact_plane,
                     float* out_z, float* out_quat, int32_t* out_nearest, cudaStream_t s) {
    if (n <= 0) return;
    const long long blocks = (n + kInitThreads - 1) / kInitThreads;
    launch_pdl(init_k, dim3((unsigned)blocks), dim3(kInitThreads), 0, s, grid_xy, n, poses_dev, n_poses, exact_plane, out_z, out_quat,
                                                     out_nearest);
    note_launches(1);
}

}  // namespace rogs
