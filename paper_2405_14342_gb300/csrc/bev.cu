// bev.cu -- stitching of chunked BEV renders (supplementary "Orthogonal
// Rendering Acceleration": a large BEV image is rendered as a grid of
// orthographic chunk cameras and the chunks are put side by side).
//
// stitch_k copies the planes of a batch of chunk views (each view's
// [3 + C + 1][h][w] planes, views back to back as the forward writes them)
// into their places of the full [3 + C + 1][H][W] image; one thread per
// (plane, row, column) of the batch, rows of a view are contiguous on both
// sides, so loads and stores are coalesced.
#include "kernels.h"

namespace rogs {

__global__ void __launch_bounds__(256) stitch_k(StitchViews sv, int n_views, int nch, const float* __restrict__ out,
                                                float* __restrict__ image, int W, int H) {
    pdl_wait();   // after the previous kernel of the stream (programmatic launch)
    const long long total = sv.pix_end[n_views - 1] * (long long)nch;
    for (long long k = blockIdx.x * 256ll + threadIdx.x; k < total; k += (long long)gridDim.x * 256) {
        // view of element k: views are laid out [view][plane][pixel]
        int v = 0;
        while (k >= sv.pix_end[v] * (long long)nch) ++v;
        const long long base = (v ? sv.pix_end[v - 1] : 0) * (long long)nch;
        const int w = sv.w[v], h = sv.h[v];
        const long long e = k - base;
        const long long plane = e / ((long long)w * h);
        const long long q = e - plane * w * h;
        const int y = (int)(q / w), x = (int)(q - (long long)y * w);
        image[(plane * H + (sv.y0[v] + y)) * (long long)W + sv.x0[v] + x] = out[k];
    }
}

void stitch_views(const StitchViews& sv, int n_views, int nch, const float* out, float* image, int W, int H,
                  cudaStream_t s) {
    const long long total = sv.pix_end[n_views - 1] * (long long)nch;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    launch_pdl(stitch_k, dim3((int)blocks), dim3(256), 0, s, sv, n_views, nch, out, image, W, H);
    note_launches(1);
}

}  // namespace rogs
