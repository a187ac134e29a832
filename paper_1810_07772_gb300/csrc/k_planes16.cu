// The 16-bit operand planes of the rank-k update (the FP16 / BF16 hi+lo split of Sec. 4.1's pair
// densities f_vc(r) = conj(psi_v(r)) psi_c(r) sqrt(2 / (E_c - E_v)), Eq. fdef, in the chunked
// K-major layout that herk16_kernel streams), the power-of-two scale that keeps FP16 in range,
// and the same planes made from any complex64 matrix (the g-space route's sphere transforms).
#include <cuda_bf16.h>
#include <algorithm>
#include <cuda_fp16.h>

#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int KC16 = HERK16_KC;
constexpr int NPL = HERK16_NPL;  // global planes per chunk
// Bound on max |f| for the FP16 scale: per r, max_v |psi_v(r)| * max_c |psi_c(r)|.
__global__ void f_bound_kernel(const float2 *__restrict__ psiT, int nr, int nb, int nv, unsigned *bound_bits)
{
    // one warp per r: the lanes read the row of psiT coalesced and reduce its two maxima
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    float best = 0.f;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < nr; r += gridDim.x * wpb) {
        float mv = 0.f, mc = 0.f;
        for (int n = lane; n < nb; n += 32) {
            const float2 z = psiT[(size_t)r * nb + n];
            const float a = sqrtf(z.x * z.x + z.y * z.y);
            if (n < nv)
                mv = fmaxf(mv, a);
            else
                mc = fmaxf(mc, a);
        }
        for (int o = 16; o > 0; o >>= 1) {
            mv = fmaxf(mv, __shfl_xor_sync(0xffffffffu, mv, o));
            mc = fmaxf(mc, __shfl_xor_sync(0xffffffffu, mc, o));
        }
        best = fmaxf(best, mv * mc);
    }
    if (lane == 0)
        atomicMax(bound_bits, __float_as_uint(best));  // non-negative floats order like their bits
}

// scale exponent e with (bound * sw_max) * 2^e <= 2^14 (FP16 max is 65504, so a factor of four
// of headroom covers any rounding in the bound); 0 for BF16, which has FP32's exponent range.
__global__ void scale_exp_kernel(const unsigned *bound_bits, float sw_max, int bf16, int *scale_exp)
{
    const float b = __uint_as_float(*bound_bits) * sw_max * 1.001f;
    int e = 0;
    if (!bf16 && b > 0.f && isfinite(b))
        e = (int)floorf(14.0f - log2f(b));
    *scale_exp = max(-100, min(100, e));
}

template <bool BF16>
__device__ __forceinline__ uint16_t to16(float x)
{
    if (BF16) {
        __nv_bfloat16 h = __float2bfloat16_rn(x);
        return *reinterpret_cast<uint16_t *>(&h);
    } else {
        __half h = __float2half_rn(x);
        return *reinterpret_cast<uint16_t *>(&h);
    }
}

template <bool BF16>
__device__ __forceinline__ float from16(uint16_t u)
{
    if (BF16) {
        __nv_bfloat16 h = *reinterpret_cast<__nv_bfloat16 *>(&u);
        return __bfloat162float(h);
    } else {
        __half h = *reinterpret_cast<__half *>(&u);
        return __half2float(h);
    }
}

// hi = rn16(x), lo = rn16(x - hi) for two values at once, packed two per word (x0 in the low half)
template <bool BF16>
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    if (BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __half2 h = __floats2half2_rn(x0, x1);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}

// The 16-bit operand planes of the pair densities.  blockIdx.y is one 16-wide chunk of k, whose
// (v, c) pairs and weights are resolved once in shared memory; threads run over the chunk in the
// order it is stored (32-bit index arithmetic, no division per element), so every warp writes
// 64 contiguous bytes per plane and reads psi_c(r) for 8 consecutive c of each r.  Used when the
// rows of psiT are too long for pair_density16_rows_kernel.
template <bool BF16>
__global__ void __launch_bounds__(256) pair_density16_kernel(const float2 *__restrict__ psiT,
                                                             const float *__restrict__ sw, int nr, int nb, int nv,
                                                             int nc, int kpad, int nr_pad, int npl,
                                                             const int *__restrict__ scale_exp,
                                                             uint16_t *__restrict__ F)
{
    __shared__ int s_v[KC16], s_c[KC16];
    __shared__ float s_w[KC16];
    const int kc = blockIdx.y;
    if (threadIdx.x < KC16) {
        const int k = kc * KC16 + threadIdx.x;
        const float s = ldexpf(1.0f, *scale_exp);
        if (k < nv * nc) {
            const int v = k / nc;
            s_v[threadIdx.x] = v;
            s_c[threadIdx.x] = nv + (k - v * nc);
            s_w[threadIdx.x] = sw[k] * s;
        } else {
            s_v[threadIdx.x] = 0;
            s_c[threadIdx.x] = 0;
            s_w[threadIdx.x] = 0.f;  // padding k: zero operand
        }
    }
    __syncthreads();
    const int per_chunk = nr_pad * KC16, nblk = nr_pad / 128;
    // plane slots: four planes Im hi, Re hi, Im lo, Re lo; six add -Im hi, -Im lo (Im hi, Im lo,
    // Re hi, Re lo first)
    const int s_rh = npl == 6 ? P6_RH : P4_RH, s_rl = npl == 6 ? P6_RL : P4_RL;
    const int s_ih = npl == 6 ? P6_IH : P4_IH, s_il = npl == 6 ? P6_IL : P4_IL;
    for (int rem = blockIdx.x * blockDim.x + threadIdx.x; rem < per_chunk; rem += gridDim.x * blockDim.x) {
        const int r = (rem >> 7) * 8 + ((rem & 63) >> 3);  // 8-row group, row in the group
        const int kk = ((rem & 127) >> 6) * 8 + (rem & 7);  // 16-byte core matrix along k, element
        float fr = 0.f, fi = 0.f;
        const float w = s_w[kk];
        if (r < nr && w != 0.f) {
            const float2 a = psiT[(size_t)r * nb + s_v[kk]];
            const float2 b = psiT[(size_t)r * nb + s_c[kk]];
            fr = fmaf(a.x, b.x, a.y * b.y) * w;   // conj(psi_v) psi_c
            fi = fmaf(a.x, b.y, -a.y * b.x) * w;
        }
        const uint16_t rh = to16<BF16>(fr), ih = to16<BF16>(fi), il = to16<BF16>(fi - from16<BF16>(ih));
        uint16_t *Fb = F + plane16_block(kc, rem >> 11, nblk, npl, 0) + (rem & 2047);
        Fb[s_rh * 2048] = rh;
        Fb[s_rl * 2048] = to16<BF16>(fr - from16<BF16>(rh));
        Fb[s_ih * 2048] = ih;
        Fb[s_il * 2048] = il;
        if (npl == 6) {  // the negated Im planes: the sign bit flipped, exact for FP16 and BF16
            Fb[P6_NIH * 2048] = ih ^ 0x8000u;
            Fb[P6_NIL * 2048] = il ^ 0x8000u;
        }
    }
}

// The same planes with the rows of psiT staged in shared memory: blockIdx.x is one 8-row group
// (its 8 rows of psiT, nb states each, read from global memory once), blockIdx.y one of
// gridDim.y parts of the k chunks.  Warp w takes chunks w, w + 8, ... of the part; each lane
// makes four consecutive k of one r (the element values are those of pair_density16_kernel, bit
// for bit) and stores 8 bytes per plane, so a warp writes the group's 256 contiguous bytes of
// every plane of a chunk.
constexpr int PD_LDP_PAD = 2;  // row pitch nb + 2 float2: lanes on 8 rows spread over the banks

template <bool BF16>
__global__ void __launch_bounds__(256) pair_density16_rows_kernel(const float2 *__restrict__ psiT,
                                                                  const float *__restrict__ sw, int nr, int nb,
                                                                  int nv, int nc, int kpad, int nr_pad, int npl,
                                                                  const int *__restrict__ scale_exp,
                                                                  uint16_t *__restrict__ F)
{
    extern __shared__ __align__(16) uint8_t smem[];
    float2 *s_psi = reinterpret_cast<float2 *>(smem);  // [8][nb + PD_LDP_PAD]
    const int ldp = nb + PD_LDP_PAD;
    const int grp = blockIdx.x;
    for (int t = threadIdx.x; t < 8 * nb; t += blockDim.x) {
        const int rr = t / nb, n = t - rr * nb, r = grp * 8 + rr;
        s_psi[rr * ldp + n] = r < nr ? psiT[(size_t)r * nb + n] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float s = ldexpf(1.0f, *scale_exp);
    const int nk = nv * nc, nchunks = kpad / KC16, nblk = nr_pad / 128;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rem = 4 * lane;                                    // element offset in the group's 128
    const int r8 = (rem & 63) >> 3, kk0 = ((rem & 127) >> 6) * 8 + (rem & 7);
    const bool live = grp * 8 + r8 < nr;
    const float2 *row = s_psi + r8 * ldp;
    const int per_part = (nchunks + gridDim.y - 1) / gridDim.y;
    const int kc_end = min(nchunks, (int)(blockIdx.y + 1) * per_part);
    for (int kc = blockIdx.y * per_part + warp; kc < kc_end; kc += 8) {
        const int k0 = kc * KC16 + kk0;
        int v = k0 / nc, c = k0 - v * nc;
        float fr[4], fi[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = k0 + i;
            fr[i] = 0.f;
            fi[i] = 0.f;
            const float w = k < nk ? sw[k] * s : 0.f;  // padding k: zero operand
            if (live && w != 0.f) {
                const float2 a = row[v];
                const float2 b = row[nv + c];
                fr[i] = fmaf(a.x, b.x, a.y * b.y) * w;   // conj(psi_v) psi_c
                fi[i] = fmaf(a.x, b.y, -a.y * b.x) * w;
            }
            if (++c == nc) {
                c = 0;
                ++v;
            }
        }
        // planes Re hi, Re lo, Im hi, Im lo, two elements per word (element i in the low half):
        // the paired conversions round each value as the single ones do
        uint32_t p[4][2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int i = 2 * j;
            split2<BF16>(fr[i], fr[i + 1], p[0][j], p[1][j]);
            split2<BF16>(fi[i], fi[i + 1], p[2][j], p[3][j]);
        }
        // the group's 128 elements in each plane of its 128-row block (slots as in
        // pair_density16_kernel)
        uint16_t *dst = F + plane16_block(kc, grp >> 4, nblk, npl, 0) + (size_t)(grp & 15) * 128 + rem;
        const int slot[4] = {npl == 6 ? P6_RH : P4_RH, npl == 6 ? P6_RL : P4_RL, npl == 6 ? P6_IH : P4_IH,
                             npl == 6 ? P6_IL : P4_IL};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint2 *>(dst + (size_t)slot[q] * 2048) = make_uint2(p[q][0], p[q][1]);
        if (npl == 6) {  // the negated Im planes: the sign bits flipped, exact for FP16 and BF16
            *reinterpret_cast<uint2 *>(dst + (size_t)P6_NIH * 2048) = make_uint2(p[2][0] ^ 0x80008000u, p[2][1] ^ 0x80008000u);
            *reinterpret_cast<uint2 *>(dst + (size_t)P6_NIL * 2048) = make_uint2(p[3][0] ^ 0x80008000u, p[3][1] ^ 0x80008000u);
        }
    }
}

// max |M[k][j]| over a complex64 matrix (rows x cols, row stride ld), as float bits.
__global__ void absmax_c64_kernel(const float2 *__restrict__ M, int rows, int cols, long ld, unsigned *bound_bits)
{
    float best = 0.f;
    const size_t total = (size_t)rows * cols;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int k = static_cast<int>(i / cols), j = static_cast<int>(i - (size_t)k * cols);
        const float2 z = M[(size_t)k * ld + j];
        best = fmaxf(best, sqrtf(z.x * z.x + z.y * z.y));
    }
    for (int o = 16; o > 0; o >>= 1)
        best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(bound_bits, __float_as_uint(best));
}

// The 16-bit hi/lo planes of a complex64 matrix M[k][j] (k < rows, j < cols), in the operand
// layout of herk16_kernel with the column index j in the place of r: row k of M is one "pair
// density" of the rank-k update, scaled by 2^scale_exp and split as pair_density16_kernel does.
template <bool BF16>
__global__ void planes16_from_c64_kernel(const float2 *__restrict__ M, int rows, int cols, long ld, int kpad,
                                         int cols_pad, const int *__restrict__ scale_exp, uint16_t *__restrict__ F)
{
    const float s = ldexpf(1.0f, *scale_exp);
    const size_t per_chunk = (size_t)cols_pad * KC16;
    const size_t total = (size_t)(kpad / KC16) * per_chunk;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t kc = i / per_chunk;
        const int rem = static_cast<int>(i - kc * per_chunk);
        const int j = (rem >> 7) * 8 + ((rem & 63) >> 3);
        const int k = static_cast<int>(kc) * KC16 + ((rem & 127) >> 6) * 8 + (rem & 7);
        float fr = 0.f, fi = 0.f;
        if (j < cols && k < rows) {
            const float2 z = M[(size_t)k * ld + j];
            fr = z.x * s;
            fi = z.y * s;
        }
        const uint16_t rh = to16<BF16>(fr), ih = to16<BF16>(fi), il = to16<BF16>(fi - from16<BF16>(ih));
        uint16_t *base = F + plane16_block((int)kc, rem >> 11, cols_pad / 128, NPL, 0) + (rem & 2047);
        base[P4_RH * 2048] = rh;
        base[P4_RL * 2048] = to16<BF16>(fr - from16<BF16>(rh));
        base[P4_IH * 2048] = ih;
        base[P4_IL * 2048] = il;
    }
}

int grid_for(size_t n)
{
    size_t g = (n + 255) / 256;
    if (g > 152 * 16)
        g = 152 * 16;
    return g < 1 ? 1 : static_cast<int>(g);
}

}  // namespace

cudaError_t launch_pair_density16(const float2 *psiT, const float *sw, float sw_max, int nr, int nb, int nv, int nc,
                                  int kpad, int nr_pad, bool bf16, unsigned *bound_bits, int *scale_exp, uint16_t *F,
                                  cudaStream_t s, int npl)
{
    if (npl != 4 && npl != 6)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(bound_bits, 0, sizeof(unsigned), s);
    if (e != cudaSuccess)
        return e;
    f_bound_kernel<<<std::max(1, std::min((nr + 7) / 8, 152 * 16)), 256, 0, s>>>(psiT, nr, nb, nv, bound_bits);
    count_launches(1);
    scale_exp_kernel<<<1, 1, 0, s>>>(bound_bits, sw_max, bf16 ? 1 : 0, scale_exp);
    count_launches(1);
    const int nchunks = kpad / KC16, per_chunk = nr_pad * KC16;
    const size_t rows_smem = (size_t)8 * (nb + PD_LDP_PAD) * sizeof(float2);
    if (rows_smem <= 100 * 1024) {
        // parts of k per row group: about 4 blocks per SM-resident slot, at least one chunk per warp
        const int ngrp = nr_pad / 8;
        const int parts = std::max(1, std::min((nchunks + 7) / 8, (152 * 6 * 4 + ngrp - 1) / ngrp));
        const dim3 g2(ngrp, parts);
        e = bf16 ? cudaFuncSetAttribute(pair_density16_rows_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)rows_smem)
                 : cudaFuncSetAttribute(pair_density16_rows_kernel<false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem);
        if (e != cudaSuccess)
            return e;
        if (bf16)
            pair_density16_rows_kernel<true><<<g2, 256, rows_smem, s>>>(psiT, sw, nr, nb, nv, nc, kpad, nr_pad,
                                                                        npl, scale_exp, F);
        else
            pair_density16_rows_kernel<false><<<g2, 256, rows_smem, s>>>(psiT, sw, nr, nb, nv, nc, kpad, nr_pad,
                                                                         npl, scale_exp, F);
        count_launches(1);
        return cudaGetLastError();
    }
    dim3 grid(std::max(1, std::min((per_chunk + 255) / 256, (152 * 16 + nchunks - 1) / nchunks)), nchunks);
    if (bf16)
        pair_density16_kernel<true><<<grid, 256, 0, s>>>(psiT, sw, nr, nb, nv, nc, kpad, nr_pad, npl, scale_exp, F);
    else
        pair_density16_kernel<false><<<grid, 256, 0, s>>>(psiT, sw, nr, nb, nv, nc, kpad, nr_pad, npl, scale_exp, F);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_planes16_from_c64(const float2 *M, int rows, int cols, long ld, int kpad, int cols_pad, bool bf16,
                                     unsigned *bound_bits, int *scale_exp, uint16_t *F, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bound_bits, 0, sizeof(unsigned), s);
    if (e != cudaSuccess)
        return e;
    absmax_c64_kernel<<<grid_for((size_t)rows * cols), 256, 0, s>>>(M, rows, cols, ld, bound_bits);
    count_launches(1);
    scale_exp_kernel<<<1, 1, 0, s>>>(bound_bits, 1.0f, bf16 ? 1 : 0, scale_exp);
    count_launches(1);
    const size_t total = (size_t)kpad * cols_pad;
    if (bf16)
        planes16_from_c64_kernel<true><<<grid_for(total), 256, 0, s>>>(M, rows, cols, ld, kpad, cols_pad, scale_exp, F);
    else
        planes16_from_c64_kernel<false><<<grid_for(total), 256, 0, s>>>(M, rows, cols, ld, kpad, cols_pad, scale_exp,
                                                                        F);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gw
