// States given as plane-wave coefficients (the DFT input of Sec. 4.1): the transform of each
// periodic part to the real-space grid,
//     u_n(r_j) = N_r^(-1/2) sum_g c_n(g) exp(+2 pi i (m1 j1/n1 + m2 j2/n2 + m3 j3/n3)),
// the discrete form of the paper's u(x) = sum_g u~(g) e^{i g.x} / sqrt(Omega) (unit-norm
// coefficient vectors give unit-norm states on the grid).  The coefficients are scattered into
// the n1 x n2 x n3 grid of Miller indices (taken modulo n) and transformed one axis at a time by
// direct DFTs with FP64-derived twiddles, in FP32 like the states the path stores.
#include <algorithm>
#include <cmath>

#include "gw_internal.cuh"

namespace gw {

namespace {

// C[b][idx[p]] = coef[b][p] (C zeroed beforehand); one block row per state.
__global__ void scatter_coef_kernel(const float2 *__restrict__ coef, int npw, const int *__restrict__ idx, int nr,
                                    float2 *__restrict__ C)
{
    const int b = blockIdx.y;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npw; p += gridDim.x * blockDim.x)
        C[(size_t)b * nr + idx[p]] = coef[(size_t)b * npw + p];
}

// out[b][..., j, ...] = scale sum_m in[b][..., m, ...] e^{+2 pi i m j / n} along the axis whose
// index has the given stride (n3 = 1, n2 = n3, n1 = n2 n3); tw[t] = e^{+2 pi i t / n}.
__global__ void dft_axis_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, int nr, int n, int stride,
                                const float2 *__restrict__ tw, float scale)
{
    const int b = blockIdx.y;
    const float2 *x = in + (size_t)b * nr;
    float2 *y = out + (size_t)b * nr;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        const int j = (r / stride) % n;
        const int base = r - j * stride;
        float ar = 0.f, ai = 0.f;
        int t = 0;
        for (int m = 0; m < n; ++m) {
            const float2 v = x[base + m * stride], w = tw[t];
            ar = fmaf(v.x, w.x, fmaf(-v.y, w.y, ar));
            ai = fmaf(v.x, w.y, fmaf(v.y, w.x, ai));
            t += j;
            if (t >= n)
                t -= n;
        }
        y[r] = make_float2(ar * scale, ai * scale);
    }
}

// P~ of one k-point into the running sum of Sec. 4.1's (1/N_k) sum over k:
// PG = (acc ? sum : 0) + w PG, in FP32 like P~ itself.
__global__ void kweight_kernel(float2 *__restrict__ PG, const float2 *__restrict__ sum, size_t n, float w, int acc)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float2 v = PG[i];
        v.x *= w;
        v.y *= w;
        if (acc) {
            v.x += sum[i].x;
            v.y += sum[i].y;
        }
        PG[i] = v;
    }
}

}  // namespace

cudaError_t launch_kweight(float2 *PG, const float2 *sum, size_t n, float w, bool acc, cudaStream_t s)
{
    const int grid = static_cast<int>(std::min<size_t>((n + 255) / 256, 152 * 8));
    kweight_kernel<<<std::max(1, grid), 256, 0, s>>>(PG, sum, n, w, acc ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

// coef: [nb][npw] complex64 (device); idx: [npw] linear grid index of each Miller index (device);
// tw: [n1 | n2 | n3] twiddle tables (device); work: nb * nr complex64; out: [nb][nr] complex64.
cudaError_t launch_states_from_g(const float2 *coef, int nb, int npw, const int *idx, int n1, int n2, int n3,
                                 const float2 *tw, float2 *work, float2 *out, cudaStream_t s)
{
    const int nr = n1 * n2 * n3;
    cudaError_t e = cudaMemsetAsync(work, 0, (size_t)nb * nr * sizeof(float2), s);
    if (e != cudaSuccess)
        return e;
    const float scale = static_cast<float>(1.0 / std::sqrt(static_cast<double>(nr)));
    for (int b0 = 0; b0 < nb; b0 += 65535) {  // grid y is one state per row, at most 65535
        const int nbb = std::min(65535, nb - b0);
        const size_t off = (size_t)b0 * nr;
        const dim3 gs((npw + 255) / 256, nbb);
        scatter_coef_kernel<<<gs, 256, 0, s>>>(coef + (size_t)b0 * npw, npw, idx, nr, work + off);
        const dim3 g((nr + 255) / 256, nbb);
        dft_axis_kernel<<<g, 256, 0, s>>>(work + off, out + off, nr, n3, 1, tw + n1 + n2, 1.0f);   // m3 -> j3
        dft_axis_kernel<<<g, 256, 0, s>>>(out + off, work + off, nr, n2, n3, tw + n1, 1.0f);       // m2 -> j2
        dft_axis_kernel<<<g, 256, 0, s>>>(work + off, out + off, nr, n1, n2 * n3, tw, scale);      // m1 -> j1
        count_launches(4);
    }
    return cudaGetLastError();
}

}  // namespace gw
