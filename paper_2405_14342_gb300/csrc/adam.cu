// adam.cu -- one fused Adam step over several parameter tensors.
//
// RoGs Sec. 4.2 optimises every surfel attribute (z only of the position),
// the colours, semantics and the exposure with Adam and per-tensor learning
// rates.  One launch covers all groups: the flat index space is the
// concatenation of the groups, each thread walks it grid-stride (coalesced
// within a group) and finds its group from the prefix offsets.  Per element:
//   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
//   p <- p - lr (m c1) / (sqrt(v c2) + eps),  c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
// and optionally g <- 0 for the next backward, which adds into it.  The
// step is bound by HBM: 16 bytes read and 12 (16 with the zeroing) written per
// element.
#include "kernels.h"

namespace rogs {

struct AdamArgs {
    rogs_adam_group g[ROGS_MAX_ADAM_GROUPS];
    long long pre[ROGS_MAX_ADAM_GROUPS + 1];   // prefix offsets of the groups in the flat index space
    int n_groups;
    float b1, b2, eps, c1, c2;
    int zero_grad;
};

__global__ void __launch_bounds__(256) adam_k(AdamArgs a) {
    const long long total = a.pre[a.n_groups];
    int gi = 0;
    for (long long k = blockIdx.x * 256ll + threadIdx.x; k < total; k += (long long)gridDim.x * 256) {
        while (k >= a.pre[gi + 1]) ++gi;   // k only grows, so the group index only moves forward
        const rogs_adam_group& G = a.g[gi];
        const long long e = k - a.pre[gi];
        const long long pi = e * (long long)G.stride;
        const float g = G.grad[pi];
        const float m = fmaf(a.b1, G.m[e], (1.0f - a.b1) * g);
        const float v = fmaf(a.b2, G.v[e], (1.0f - a.b2) * g * g);
        G.m[e] = m;
        G.v[e] = v;
        G.param[pi] -= G.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
        if (a.zero_grad) G.grad[pi] = 0.0f;
    }
}

void adam_step(const rogs_adam_group* groups, int n_groups, int step, float b1, float b2, float eps, bool zero_grad,
               cudaStream_t s) {
    AdamArgs a{};
    a.n_groups = n_groups;
    a.pre[0] = 0;
    for (int i = 0; i < n_groups; ++i) {
        a.g[i] = groups[i];
        a.pre[i + 1] = a.pre[i] + groups[i].n;
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
    adam_k<<<(int)blocks, 256, 0, s>>>(a);
    note_launches(1);
}

}  // namespace rogs
