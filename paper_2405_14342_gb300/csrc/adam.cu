// adam.cu -- one fused Adam step over several parameter tensors.
//
// RoGs Sec. 4.2 optimises every surfel attribute (z only of the position),
// the colours, semantics and the exposure with Adam and per-tensor learning
// rates.  One launch covers all groups: the flat index space is the
// concatenation of the groups' 4-element chunks, each thread walks it
// grid-stride (coalesced within a group, float4 where a group is contiguous
// and aligned) and finds its group from the prefix offsets.  Per element:
//   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
//   p <- p - lr (m c1) / (sqrt(v c2) + eps),  c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
// and optionally g <- 0 for the next backward, which adds into it (with the
// group's zero_lead floats before g: the x and y gradients of the z column,
// which Sec. 4.2 does not learn).  Each group's learning rate for this step
// (constant, or z's log-linear decay from lr to lr_end) is evaluated on the
// host in double before the launch.  The step is bound by HBM: 16 bytes read and 12 (16 with the zeroing) written per
// element.
#include <algorithm>

#include "kernels.h"

namespace rogs {

struct AdamArgs {
    rogs_adam_group g[ROGS_MAX_ADAM_GROUPS];
    long long pre[ROGS_MAX_ADAM_GROUPS + 1];   // prefix offsets of the groups, in 4-element chunks
    int vec[ROGS_MAX_ADAM_GROUPS];             // stride 1 and all four arrays 16-byte aligned
    int n_groups;
    float b1, b2, eps, c1, c2;
    int zero_grad;
};

__device__ __forceinline__ void adam_one(const AdamArgs& a, float& p, float& g, float& m, float& v, float lr) {
    m = fmaf(a.b1, m, (1.0f - a.b1) * g);
    v = fmaf(a.b2, v, (1.0f - a.b2) * g * g);
    p -= lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
    if (a.zero_grad) g = 0.0f;
}

// One thread per 4-element chunk of a group (grid-stride over all chunks):
// float4 loads and stores where the group allows them, else four scalars.
__global__ void __launch_bounds__(256) adam_k(AdamArgs a) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    const long long total = a.pre[a.n_groups];
    int gi = 0;
    for (long long k = blockIdx.x * 256ll + threadIdx.x; k < total; k += (long long)gridDim.x * 256) {
        while (k >= a.pre[gi + 1]) ++gi;   // k only grows, so the group index only moves forward
        const rogs_adam_group& G = a.g[gi];
        const long long e0 = 4 * (k - a.pre[gi]);
        if (a.vec[gi] && e0 + 4 <= G.n) {
            float4 p = reinterpret_cast<float4*>(G.param)[e0 / 4];
            float4 g = reinterpret_cast<float4*>(G.grad)[e0 / 4];
            float4 m = reinterpret_cast<float4*>(G.m)[e0 / 4];
            float4 v = reinterpret_cast<float4*>(G.v)[e0 / 4];
            adam_one(a, p.x, g.x, m.x, v.x, G.lr);
            adam_one(a, p.y, g.y, m.y, v.y, G.lr);
            adam_one(a, p.z, g.z, m.z, v.z, G.lr);
            adam_one(a, p.w, g.w, m.w, v.w, G.lr);
            reinterpret_cast<float4*>(G.param)[e0 / 4] = p;
            reinterpret_cast<float4*>(G.m)[e0 / 4] = m;
            reinterpret_cast<float4*>(G.v)[e0 / 4] = v;
            if (a.zero_grad) reinterpret_cast<float4*>(G.grad)[e0 / 4] = g;
        } else {
            for (long long e = e0; e < e0 + 4 && e < G.n; ++e) {
                const long long pi = e * (long long)G.stride;
                float p = G.param[pi], g = G.grad[pi], m = G.m[e], v = G.v[e];
                adam_one(a, p, g, m, v, G.lr);
                G.param[pi] = p;
                G.m[e] = m;
                G.v[e] = v;
                if (a.zero_grad) {
                    G.grad[pi] = g;
                    for (int j = 1; j <= G.zero_lead; ++j) G.grad[pi - j] = 0.0f;
                }
            }
        }
    }
}

void adam_step(const rogs_adam_group* groups, int n_groups, int step, float b1, float b2, float eps, bool zero_grad,
               cudaStream_t s) {
    AdamArgs a{};
    a.n_groups = n_groups;
    a.pre[0] = 0;
    auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
    for (int i = 0; i < n_groups; ++i) {
        const rogs_adam_group& g = groups[i];
        a.g[i] = g;
        if (g.decay_steps > 0) {   // lr_t = lr (lr_end / lr)^min((t - 1) / decay_steps, 1)
            const double f = std::min(1.0, (double)(step - 1) / (double)g.decay_steps);
            a.g[i].lr = (float)((double)g.lr * std::pow((double)g.lr_end / (double)g.lr, f));
        }
        a.pre[i + 1] = a.pre[i] + (g.n + 3) / 4;
        a.vec[i] = g.stride == 1 && g.zero_lead == 0 && al16(g.param) && al16(g.grad) && al16(g.m) && al16(g.v);
    }
    a.b1 = b1;
    a.b2 = b2;
    a.eps = eps;
    a.c1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)step)));
    a.c2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)step)));
    a.zero_grad = zero_grad ? 1 : 0;
    const long long total = a.pre[n_groups];
    if (total == 0) return;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    launch_pdl(adam_k, dim3((int)blocks), dim3(256), 0, s, a);
    note_launches(1);
}

}  // namespace rogs
