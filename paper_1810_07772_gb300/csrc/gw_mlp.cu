// Learned truncation correction of P~(G,G').
//
// The sum over unoccupied states c in Eq. (Pstatic) is cut at some N_c in practice, and the paper
// lists this band truncation among the costs of the method (Sec. 2) without prescribing a cure.
// This file adds one: a multilayer perceptron maps per-entry features of the truncated P~ to the
// missing part P~(N_c = all) - P~(N_c = kept).  Everything runs on the device:
//
//   features / targets / apply   element-wise kernels over the upper triangle of P~
//   forward / backward           the products with 256-wide (hidden) sides on the tensor cores
//                                (k_mlp_train.cu: FP32 operands as three BF16 parts, FP32
//                                accuracy; bias + tanh and tanh' in the epilogues; the weight
//                                gradients over slices of the batch, added in a fixed order);
//                                the 2-wide output layer, the loss, the deltas of layer 3 and
//                                the output layer's gradient in one kernel (a warp per row, sums
//                                per block added in a fixed order); the weights are the
//                                FP16-rounded ones
//   loss                         L = (1 / (2B)) sum (y - t)^2 and dL/dy = (y - t) / B
//   optimiser                    Adam on an FP32 master copy; the FP16 weights are rounded from it
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include <cooperative_groups.h>
#include <cub/cub.cuh>

#include "gw_internal.cuh"

namespace gw {
void count_launches(int n);
}

namespace {

constexpr int NF = 12;        // features per P~ entry
constexpr int NOUT = 2;       // (Re, Im) of the predicted correction
constexpr int SPLIT_MAX = 64;

// Position of entry (g, h), g <= h, in the row-major upper triangle of an ng x ng matrix.
__device__ __forceinline__ long tri_index(int g, int h, int ng)
{
    return (long)g * ng - (long)g * (g - 1) / 2 + (h - g);
}

// ---------------------------------------------------------------------------------------------
// Per-system scalars

// ratio = sum_{c >= keep} sum_v 2/(E_c - E_v)  /  sum_{c < keep} sum_v 2/(E_c - E_v)   (FP64)
// FP64 runs at a small fraction of the FP32 rate on this GPU, so the nv nc_all terms are spread
// over one cluster of RATIO_CLUSTER blocks, a thread per unoccupied state c at a time (the
// occupied energies in each block's shared memory).  1/d is the hardware FP32 reciprocal
// approximation (relative error ~2^-23, seeded with d rounded to FP32) refined by one FP64
// Newton-Raphson step r <- r + r (1 - d r), which squares the relative error to ~2^-45, instead of
// an FP64 division per term.  The blocks' partial sums are added by block 0 through distributed
// shared memory in rank order, so the result does not depend on scheduling.
constexpr int RATIO_THREADS = 512;
constexpr int RATIO_CLUSTER = 8;
constexpr int RATIO_MAX_NV = 1024;

__device__ __forceinline__ double recip_nr(double d)
{
    if (!(fabs(d) > 1e-30 && fabs(d) < 1e30))  // outside the FP32 seed's normal range
        return 1.0 / d;
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"((float)d));
    const double r = (double)r0;
    return fma(r, fma(-d, r, 1.0), r);
}

__global__ void __cluster_dims__(RATIO_CLUSTER, 1, 1) __launch_bounds__(RATIO_THREADS)
    weight_ratio_kernel(const double *E, int nv, int keep, int nc_all, float *ratio)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ double ev[RATIO_MAX_NV];
    __shared__ double s_om[RATIO_THREADS / 32], s_in[RATIO_THREADS / 32];
    __shared__ double part[2];
    for (int v = threadIdx.x; v < nv; v += RATIO_THREADS)
        ev[v] = E[v];
    __syncthreads();
    double om = 0, in = 0;
    for (int c = (int)cluster.block_rank() * RATIO_THREADS + threadIdx.x; c < nc_all;
         c += RATIO_THREADS * RATIO_CLUSTER) {
        const double ec = E[nv + c];
        double acc = 0;
        for (int v = 0; v < nv; ++v)
            acc += recip_nr(ec - ev[v]);
        if (c < keep)
            in += 2.0 * acc;
        else
            om += 2.0 * acc;
    }
    for (int o = 16; o > 0; o >>= 1) {
        om += __shfl_xor_sync(0xffffffffu, om, o);
        in += __shfl_xor_sync(0xffffffffu, in, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_om[warp] = om;
        s_in[warp] = in;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w = 0; w < RATIO_THREADS / 32; ++w) {
            a += s_om[w];
            b += s_in[w];
        }
        part[0] = a;
        part[1] = b;
    }
    cluster.sync();  // every block's partial sums are written
    if (cluster.block_rank() == 0 && threadIdx.x == 0) {
        double a = 0, b = 0;
        for (unsigned r = 0; r < RATIO_CLUSTER; ++r) {
            const double *p = cluster.map_shared_rank(part, r);
            a += p[0];
            b += p[1];
        }
        *ratio = (float)(a / b);
    }
    cluster.sync();  // the other blocks keep their shared memory until block 0 has read it
}

// s = 1 / mean_{g >= 1} |Re P~(g, g)|  (FP64 sum)
__global__ void __launch_bounds__(256) entry_scale_kernel(const float2 *PG, int ng, float *scale)
{
    __shared__ double red[256];
    double acc = 0;
    for (int g = 1 + threadIdx.x; g < ng; g += blockDim.x)
        acc += fabs((double)PG[(long)g * ng + g].x);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *scale = red[0] > 0 ? (float)((double)(ng - 1) / red[0]) : 0.f;
}

// One block per row g; threads over h in [g, ng).
__global__ void __launch_bounds__(128) features_kernel(const float2 *PG, int ng, const int *gvec, float inv_gcut,
                                                       const float *ratio, const float2 *clos, const float *scale,
                                                       float *X)
{
    const int g = blockIdx.x;
    const float s = *scale, rt = *ratio;
    const int g1 = gvec[3 * g], g2 = gvec[3 * g + 1], g3 = gvec[3 * g + 2];
    const float m2g = (float)(g1 * g1 + g2 * g2 + g3 * g3);
    const float dg = PG[(long)g * ng + g].x;
    for (int h = g + (int)threadIdx.x; h < ng; h += blockDim.x) {
        const int h1 = gvec[3 * h], h2 = gvec[3 * h + 1], h3 = gvec[3 * h + 2];
        const int d1 = g1 - h1, d2 = g2 - h2, d3 = g3 - h3;
        const float2 p = PG[(long)g * ng + h];
        float *x = X + tri_index(g, h, ng) * NF;
        x[0] = m2g * inv_gcut;
        x[1] = (float)(h1 * h1 + h2 * h2 + h3 * h3) * inv_gcut;
        x[2] = (float)(d1 * d1 + d2 * d2 + d3 * d3) * (0.25f * inv_gcut);
        x[3] = s * p.x;
        x[4] = s * p.y;
        x[5] = s * dg;
        x[6] = s * PG[(long)h * ng + h].x;
        x[7] = g == h ? 1.f : 0.f;
        x[8] = rt;
        x[9] = (g == 0 || h == 0) ? 1.f : 0.f;
        const float2 dc = clos ? clos[(long)g * ng + h] : make_float2(0.f, 0.f);
        x[10] = s * dc.x;
        x[11] = s * dc.y;
    }
}

// t = s (hi - lo - clos)(g, h): what the closure estimate leaves (clos may be null)
__global__ void __launch_bounds__(128) targets_kernel(const float2 *lo, const float2 *hi, const float2 *clos, int ng,
                                                      const float *scale, float *T)
{
    const int g = blockIdx.x;
    const float s = *scale;
    for (int h = g + (int)threadIdx.x; h < ng; h += blockDim.x) {
        const long e = (long)g * ng + h;
        float *t = T + tri_index(g, h, ng) * NOUT;
        const float2 dc = clos ? clos[e] : make_float2(0.f, 0.f);
        t[0] = s * (hi[e].x - lo[e].x - dc.x);
        t[1] = s * (hi[e].y - lo[e].y - dc.y);
    }
}

// P~(g,h) += clos(g,h) + (y0 + i y1)/s and P~(h,g) = its conjugate; diagonal: real part only;
// row and column 0 untouched (clos may be null).
__global__ void __launch_bounds__(128) apply_kernel(float2 *PG, int ng, const float *Y, const float *scale,
                                                    const float2 *clos)
{
    const int g = blockIdx.x;
    if (g == 0)
        return;
    const float inv = 1.f / *scale;
    for (int h = g + (int)threadIdx.x; h < ng; h += blockDim.x) {
        const float *y = Y + tri_index(g, h, ng) * NOUT;
        const float2 dc = clos ? clos[(long)g * ng + h] : make_float2(0.f, 0.f);
        const float dr = y[0] * inv + dc.x, di = y[1] * inv + dc.y;
        if (h == g) {
            PG[(long)g * ng + g].x += dr;
        } else {
            float2 &a = PG[(long)g * ng + h];
            float2 &b = PG[(long)h * ng + g];
            a.x += dr;
            a.y += di;
            b.x += dr;
            b.y -= di;
        }
    }
}

// gW[e] = sum_z part[z * stride + e] (e < n_w) and, from blocks past the first nb_w,
// gb[o] = sum_rb csum[rb * out + o] (o < out, rb < nrb): both in a fixed order
__global__ void __launch_bounds__(256) grad_finish_kernel(const float *part, int S, long stride, long n_w, int nb_w,
                                                          float *gW, const float *csum, int nrb, int out, float *gb)
{
    if ((int)blockIdx.x < nb_w) {
        for (long e = blockIdx.x * 256L + threadIdx.x; e < n_w; e += (long)nb_w * 256) {
            float acc = 0.f;
            for (int z = 0; z < S; ++z)
                acc += part[z * stride + e];
            gW[e] = acc;
        }
        return;
    }
    const int o = ((int)blockIdx.x - nb_w) * 256 + threadIdx.x;
    if (o < out) {
        float acc = 0.f;
        for (int rb = 0; rb < nrb; ++rb)
            acc += csum[(long)rb * out + o];
        gb[o] = acc;
    }
}

// The 2-wide output layer, OUT_ROWS rows per block (8 warps, a warp per row at a time): y = W4 h + b4
// (h = H2[b], W4 FP16) into Y.  With targets T (row trow[b] if given) also D4[b] = (y - t) / B,
// loss += |y - t|^2 / (2B), the deltas of layer 3, D[b][n] = (D4[b] W4)[n] (1 - h[n]^2), and the
// block's share of the output layer's gradient, part[block] = [sum_b D4[b] h^T (2 x Hd) | sum_b D4[b]]
// (2 Hd + 2 values; each warp sums its rows in shared memory, the warps are then added in order).
constexpr int OUT_ROWS = 16;
// out[e] = sum_s part[s * G + e] for one e per block: strided partial sums, then a tree, both in a
// fixed order
__global__ void __launch_bounds__(256) sum_parts_tree_kernel(const float *part, int S, long G, float *out)
{
    __shared__ float red[256];
    const long e = blockIdx.x;
    float acc = 0.f;
    for (int z = threadIdx.x; z < S; z += 256)
        acc += part[z * G + e];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        out[e] = red[0];
}

__global__ void __launch_bounds__(256) out_layer_kernel(const float *H2, int Hd, const __half *W4, const float *b4,
                                                        int batch, float *Y, const float *T, const int *trow,
                                                        float invB, float *D4, float *D, float *loss, float *part)
{
    extern __shared__ float gsh[];  // [8 warps][2 Hd + 2]
    __shared__ float red[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, G = 2 * Hd + 2;
    float *g = gsh + warp * G;
    if (T)
        for (int e = lane; e < G; e += 32)
            g[e] = 0.f;
    __syncwarp();
    float l2 = 0.f, s0 = 0.f, s1 = 0.f;
    for (int rr = warp; rr < OUT_ROWS; rr += 8) {
        const int b = blockIdx.x * OUT_ROWS + rr;
        if (b >= batch)
            break;
        const float *h = H2 + (long)b * Hd;
        float y0 = 0.f, y1 = 0.f;
        for (int n = lane; n < Hd; n += 32) {
            const float hv = h[n];
            y0 = fmaf(__half2float(W4[n]), hv, y0);
            y1 = fmaf(__half2float(W4[Hd + n]), hv, y1);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            y0 += __shfl_xor_sync(0xffffffffu, y0, o);
            y1 += __shfl_xor_sync(0xffffffffu, y1, o);
        }
        y0 += b4[0];
        y1 += b4[1];
        if (lane == 0) {
            Y[2 * (long)b] = y0;
            Y[2 * (long)b + 1] = y1;
        }
        if (T) {
            const long r = trow ? trow[b] : b;
            const float e0 = y0 - T[2 * r], e1 = y1 - T[2 * r + 1];
            const float d0 = e0 * invB, d1 = e1 * invB;
            if (lane == 0) {
                D4[2 * (long)b] = d0;
                D4[2 * (long)b + 1] = d1;
            }
            l2 += e0 * e0 + e1 * e1;
            s0 += d0;
            s1 += d1;
            for (int n = lane; n < Hd; n += 32) {
                const float hv = h[n];
                const float w0 = __half2float(W4[n]), w1 = __half2float(W4[Hd + n]);
                D[(long)b * Hd + n] = (d0 * w0 + d1 * w1) * (1.f - hv * hv);
                g[n] += d0 * hv;
                g[Hd + n] += d1 * hv;
            }
        }
    }
    if (!T)
        return;
    if (lane == 0) {
        g[2 * Hd] = s0;
        g[2 * Hd + 1] = s1;
        red[warp] = l2;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < G; e += 256) {
        float acc = 0.f;
        for (int w = 0; w < 8; ++w)
            acc += gsh[w * G + e];
        part[(long)blockIdx.x * G + e] = acc;
    }
    if (threadIdx.x == 0 && loss) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w)
            t += red[w];
        atomicAdd(loss, 0.5f * invB * t);
    }
}

__global__ void adam_kernel(float *theta, __half *theta16, float *w32, const float *g, float *m, float *v, long P,
                            float lr, float b1, float b2, float c1, float c2, float eps)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < P; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float t = theta[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        theta[i] = t;
        const __half t16 = __float2half_rn(t);
        theta16[i] = t16;
        w32[i] = __half2float(t16);
    }
}

__global__ void to_half_kernel(const float *x, __half *y, float *y32, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const __half h = __float2half_rn(x[i]);
        y[i] = h;
        y32[i] = __half2float(h);
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Network state and host orchestration

struct gw_mlp {
    int device = 0, n_in = 0, hidden = 0, max_batch = 0, num_sms = 0;
    long P = 0;
    long off_w[4] = {}, off_b[4] = {};
    cudaStream_t stream = nullptr;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __half *theta16 = nullptr;
    float *H[3] = {}, *Da = nullptr, *Db = nullptr, *D4 = nullptr, *Y = nullptr, *part = nullptr;
    // tensor-core products: the FP16-rounded parameters as FP32, and the operands in the
    // three-part BF16 block layout: X, H0, H1 as layer inputs (row) and weight-gradient operands
    // (col), the deltas (row: two, a product reads one and writes the other; col), W1..W3 (row)
    // and W2, W3 transposed (col)
    float *w32 = nullptr;
    uint8_t *pX = nullptr, *pXc = nullptr, *pH[2] = {}, *pHc[2] = {}, *pD[2] = {}, *pDc = nullptr;
    uint8_t *pW[3] = {}, *pWc[2] = {};
    float *csum = nullptr;  // column sums of the deltas per 128-row tile (bias gradients)
    bool wpacked = false;
    long step = 0;
    // tensor-core inference: W1, W2, W3 in the operand layout (valid while tiled == true); d_err:
    // the status word of every tensor-core kernel's bounded waits (read by gw_mlp_check)
    uint8_t *Wt = nullptr;
    bool tiled = false;
    uint32_t *d_err = nullptr;
    std::string last_error;
};

namespace {

gw_status mfail(gw_mlp *m, gw_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (m)
        m->last_error = buf;
    return st;
}

gw_status mcuda(gw_mlp *m, cudaError_t e, const char *where)
{
    cudaGetLastError();
    return mfail(m, e == cudaErrorMemoryAllocation ? GW_E_NOMEM : GW_E_CUDA, "%s: %s", where,
                 cudaGetErrorString(e));
}

#define MLP_TRY(expr)               \
    do {                            \
        gw_status s_ = (expr);      \
        if (s_ != GW_OK)            \
            return s_;              \
    } while (0)

#define MLP_CUDA(call, where)            \
    do {                                 \
        cudaError_t e_ = (call);         \
        if (e_ != cudaSuccess)           \
            return mcuda(m, e_, where);  \
    } while (0)

long num_params(int n_in, int hidden)
{
    return (long)hidden * n_in + hidden + 2L * ((long)hidden * hidden + hidden) + (long)NOUT * hidden + NOUT;
}

constexpr uint64_t TC_WAIT_NS = 2000000000ull;

// W1..W3 as the B operands of the forward products (rows = outputs) and W2, W3 transposed for the
// products back through them (rows = inputs), from the FP16-rounded weights
cudaError_t pack_weights(gw_mlp *m)
{
    if (m->wpacked)
        return cudaSuccess;
    gw::MlpWeightPack p{};
    for (int l = 0; l < 3; ++l) {
        p.row[l] = m->pW[l];
        p.off[l] = m->off_w[l];
    }
    p.col[0] = m->pWc[0];
    p.col[1] = m->pWc[1];
    p.hidden = m->hidden;
    p.n_in = m->n_in;
    const cudaError_t e = gw::launch_mlp_pack_weights(m->w32, p, m->num_sms, m->stream);
    if (e == cudaSuccess)
        m->wpacked = true;
    return e;
}

// Forward of `batch` rows of X (gathered by rows if given) into H[0..2] and Yout.  keep: also
// pack what the backward pass needs (X and H0, H1 as weight-gradient operands).  Yout null: stop
// before the output layer.
cudaError_t forward_batch(gw_mlp *m, const float *X, const int *rows, int batch, float *Yout, bool keep)
{
    const int Hd = m->hidden;
    cudaError_t e = pack_weights(m);
    if (e == cudaSuccess)
        e = gw::launch_mlp_pack3(X, m->n_in, rows, batch, m->n_in, m->pX, keep ? m->pXc : nullptr, nullptr,
                                 m->stream);
    const uint8_t *Ain = m->pX;
    int K = m->n_in;
    // each layer also writes its output as the next layer's operand and, for the backward pass, as
    // the operand of a weight gradient
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
        e = gw::launch_mlp_gemm3(1, Ain, batch, m->pW[l], Hd, K, 1, m->H[l], Hd, 0, m->theta + m->off_b[l], nullptr, 0,
                                 l < 2 ? m->pH[l] : nullptr, keep && l < 2 ? m->pHc[l] : nullptr, nullptr, m->d_err,
                                 TC_WAIT_NS, m->stream, nullptr);
        if (l < 2) {
            Ain = m->pH[l];
            K = Hd;
        }
    }
    if (e != cudaSuccess || !Yout)
        return e;
    // the 2-wide output layer
    out_layer_kernel<<<(batch + OUT_ROWS - 1) / OUT_ROWS, 256, 0, m->stream>>>(
        m->H[2], Hd, m->theta16 + m->off_w[3], m->theta + m->off_b[3], batch, Yout, nullptr, nullptr, 0.f, nullptr,
        nullptr, nullptr, nullptr);
    gw::count_launches(1);
    return cudaGetLastError();
}

// Loss and the gradient of every parameter into m->grad.
cudaError_t loss_grad(gw_mlp *m, const float *X, const float *T, const int *rows, int batch, float *loss)
{
    const int Hd = m->hidden;
    cudaError_t e = forward_batch(m, X, rows, batch, nullptr, true);
    if (e != cudaSuccess)
        return e;
    // output layer, loss, its deltas D4 = (y - t) / B, those of layer 3, D = (D4 W4) (1 - H2^2), and
    // per-block partial sums of dW4, db4, then added over the blocks (W4 and b4 are adjacent)
    const int nob = (batch + OUT_ROWS - 1) / OUT_ROWS;
    const size_t osh = (size_t)8 * (2 * Hd + 2) * sizeof(float);
    if ((e = cudaFuncSetAttribute(out_layer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)osh)) !=
        cudaSuccess)
        return e;
    out_layer_kernel<<<nob, 256, osh, m->stream>>>(m->H[2], Hd, m->theta16 + m->off_w[3], m->theta + m->off_b[3],
                                                    batch, m->Y, T, rows, 1.f / batch, m->D4, m->Da, loss, m->part);
    gw::count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    sum_parts_tree_kernel<<<2 * Hd + 2, 256, 0, m->stream>>>(m->part, nob, 2L * Hd + 2, m->grad + m->off_w[3]);
    gw::count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    // hidden layers l = 2, 1, 0 (weights W_{l+1}): dW = D^T (layer input), db = the column sums of D,
    // and the deltas of layer l - 1, (D W_{l+1}) (1 - H_{l-1}^2), which the product writes as the
    // operands of the next steps (row, col) with their column sums
    if ((e = gw::launch_mlp_pack3(m->Da, Hd, nullptr, batch, Hd, m->pD[0], m->pDc, m->csum, m->stream)) !=
        cudaSuccess)
        return e;
    float *D = m->Da;
    int cur = 0;
    for (int l = 2; l >= 0; --l) {
        const int in = l > 0 ? Hd : m->n_in;
        const int tiles = ((Hd + 127) / 128) * ((in + 127) / 128);
        int S = 1;
        if ((e = gw::launch_mlp_gemm3(0, m->pDc, Hd, l > 0 ? m->pHc[l - 1] : m->pXc, in, batch,
                                      std::max(1, std::min(SPLIT_MAX, m->num_sms / tiles)), m->part, in,
                                      (long)Hd * in, nullptr, nullptr, 0, nullptr, nullptr, nullptr, m->d_err,
                                      TC_WAIT_NS, m->stream, &S)) != cudaSuccess)
            return e;
        const long nw = (long)Hd * in;
        const int nbw = (int)std::min<long>((nw + 255) / 256, 4L * m->num_sms);
        grad_finish_kernel<<<nbw + (Hd + 255) / 256, 256, 0, m->stream>>>(
            m->part, S, nw, nw, nbw, m->grad + m->off_w[l], m->csum, (batch + 127) / 128, Hd, m->grad + m->off_b[l]);
        gw::count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        if (l > 0) {
            float *Dn = D == m->Da ? m->Db : m->Da;
            if ((e = gw::launch_mlp_gemm3(2, m->pD[cur], batch, m->pWc[l - 1], Hd, Hd, 1, Dn, Hd, 0, nullptr,
                                          m->H[l - 1], Hd, l > 1 ? m->pD[1 - cur] : nullptr, m->pDc, m->csum, m->d_err,
                                          TC_WAIT_NS, m->stream, nullptr)) != cudaSuccess)
                return e;
            D = Dn;
            cur = 1 - cur;
        }
    }
    return cudaSuccess;
}

gw_status check_mlp(gw_mlp *m)
{
    if (!m)
        return GW_E_INVALID;
    const cudaError_t e = cudaSetDevice(m->device);
    if (e != cudaSuccess)
        return mcuda(m, e, "cudaSetDevice");
    return GW_OK;
}

}  // namespace

namespace {

// One Adam step on a batch (arguments checked by the callers).
gw_status train_step(gw_mlp *m, const float *X, const float *T, const int *rows, int batch, double lr, double beta1,
                     double beta2, double adam_eps, float *loss_accum)
{
    MLP_CUDA(loss_grad(m, X, T, rows, batch, loss_accum), "gw_mlp_train_step");
    m->step += 1;
    m->tiled = false;
    m->wpacked = false;
    const double c1 = 1.0 / (1.0 - std::pow(beta1, (double)m->step));
    const double c2 = 1.0 / (1.0 - std::pow(beta2, (double)m->step));
    adam_kernel<<<(int)std::min<long>((m->P + 255) / 256, 4L * m->num_sms), 256, 0, m->stream>>>(
        m->theta, m->theta16, m->w32, m->grad, m->m, m->v, m->P, (float)lr, (float)beta1, (float)beta2, (float)c1,
        (float)c2, (float)adam_eps);
    gw::count_launches(1);
    MLP_CUDA(cudaGetLastError(), "gw_mlp_train_step adam");
    return GW_OK;
}

// SplitMix64's output function (Steele, Lea and Flood, 2014): a bijective mix of 64 bits.
__host__ __device__ __forceinline__ unsigned long long splitmix64_mix(unsigned long long z)
{
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

// Sort key of pool position j in pass e: the minibatch order of a pass is the pool sorted by it.
__global__ void order_keys_kernel(unsigned long long seed, int pass, long S, unsigned long long *keys)
{
    const unsigned long long base = seed * 0x9E3779B97F4A7C15ull + (unsigned long long)(pass + 1) * 0xD1B54A32D192ED03ull;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < S; j += (long)gridDim.x * blockDim.x)
        keys[j] = splitmix64_mix(base + (unsigned long long)j);
}

// flags[i] = (X[i][feat] == 1), idx[i] = i
__global__ void diag_flags_kernel(const float *X, long n, int nf, int feat, unsigned char *flags, int *idx)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        flags[i] = X[i * nf + feat] == 1.0f ? 1 : 0;
        idx[i] = (int)i;
    }
}

// pool[j] = j for j < n, then the rows D[0..nd) repeated: pool[n + q] = D[q % nd]
__global__ void pool_kernel(long n, const int *D, int nd, long S, int *pool)
{
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < S; j += (long)gridDim.x * blockDim.x)
        pool[j] = j < n ? (int)j : D[(j - n) % nd];
}

int blocks_for(long n, int num_sms)
{
    return (int)std::max(1L, std::min((n + 255) / 256, 8L * num_sms));
}

}  // namespace

extern "C" {

gw_status gw_mlp_num_params(int n_in, int hidden, size_t *n)
{
    if (!n || n_in < 1 || hidden < 1)
        return GW_E_INVALID;
    *n = (size_t)num_params(n_in, hidden);
    return GW_OK;
}

gw_status gw_mlp_create(gw_mlp **out, int device, int n_in, int hidden, int max_batch, void *stream)
{
    if (!out)
        return GW_E_INVALID;
    *out = nullptr;
    if (n_in < 1 || n_in > 64 || hidden < 1 || hidden > 1024 || max_batch < 1 || max_batch > (1 << 22))
        return GW_E_INVALID;
    gw_mlp *m = new (std::nothrow) gw_mlp;
    if (!m)
        return GW_E_NOMEM;
    m->device = device;
    m->n_in = n_in;
    m->hidden = hidden;
    m->max_batch = max_batch;
    m->stream = static_cast<cudaStream_t>(stream);
    m->P = num_params(n_in, hidden);
    const long sizes[4][2] = {{hidden, n_in}, {hidden, hidden}, {hidden, hidden}, {NOUT, hidden}};
    long o = 0;
    for (int l = 0; l < 4; ++l) {
        m->off_w[l] = o;
        o += sizes[l][0] * sizes[l][1];
        m->off_b[l] = o;
        o += sizes[l][0];
    }
    auto cleanup = [&](gw_status st) {
        gw_mlp_destroy(m);
        return st;
    };
    if (cudaSetDevice(device) != cudaSuccess || cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount,
                                                                       device) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(GW_E_CUDA);
    }
    const size_t P = (size_t)m->P, act = (size_t)max_batch * hidden;
    const size_t part = std::max((size_t)SPLIT_MAX * hidden * (std::max(hidden, n_in) + 1),
                                 (size_t)((max_batch + 15) / 16) * (2 * hidden + 2));  // + output-layer partials
    float **fbufs[] = {&m->theta, &m->grad, &m->m, &m->v, &m->w32};
    for (float **p : fbufs)
        if (cudaMalloc(p, P * sizeof(float)) != cudaSuccess)
            return cleanup(GW_E_NOMEM);
    if (cudaMalloc(&m->theta16, P * sizeof(__half)) != cudaSuccess)
        return cleanup(GW_E_NOMEM);
    float **abufs[] = {&m->H[0], &m->H[1], &m->H[2], &m->Da, &m->Db};
    for (float **p : abufs)
        if (cudaMalloc(p, act * sizeof(float)) != cudaSuccess)
            return cleanup(GW_E_NOMEM);
    if (cudaMalloc(&m->D4, (size_t)max_batch * NOUT * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&m->Y, (size_t)max_batch * NOUT * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&m->part, part * sizeof(float)) != cudaSuccess)
        return cleanup(GW_E_NOMEM);
    // operands of the tensor-core products (sizes: rows x k of each)
    struct {
        uint8_t **p;
        int rows, k;
    } packs[] = {{&m->pX, max_batch, n_in},      {&m->pXc, n_in, max_batch},      {&m->pH[0], max_batch, hidden},
                 {&m->pH[1], max_batch, hidden}, {&m->pHc[0], hidden, max_batch}, {&m->pHc[1], hidden, max_batch},
                 {&m->pD[0], max_batch, hidden}, {&m->pD[1], max_batch, hidden},  {&m->pDc, hidden, max_batch},
                 {&m->pW[0], hidden, n_in},
                 {&m->pW[1], hidden, hidden},    {&m->pW[2], hidden, hidden},     {&m->pWc[0], hidden, hidden},
                 {&m->pWc[1], hidden, hidden}};
    for (auto &pk : packs)
        if (cudaMalloc(pk.p, gw::mlp_pack3_bytes(pk.rows, pk.k)) != cudaSuccess)
            return cleanup(GW_E_NOMEM);
    // the weights' padding is never written: clear their buffers once
    for (uint8_t *w : {m->pW[0], m->pW[1], m->pW[2], m->pWc[0], m->pWc[1]})
        if (cudaMemsetAsync(w, 0, gw::mlp_pack3_bytes(hidden, w == m->pW[0] ? n_in : hidden), m->stream) != cudaSuccess)
            return cleanup(GW_E_CUDA);
    if (cudaMalloc(&m->d_err, sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&m->csum, (size_t)((max_batch + 127) / 128) * hidden * sizeof(float)) != cudaSuccess)
        return cleanup(GW_E_NOMEM);
    if (cudaMemsetAsync(m->theta, 0, P * sizeof(float), m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->theta16, 0, P * sizeof(__half), m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->w32, 0, P * sizeof(float), m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->d_err, 0, sizeof(uint32_t), m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->m, 0, P * sizeof(float), m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->v, 0, P * sizeof(float), m->stream) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(GW_E_CUDA);
    }
    *out = m;
    return GW_OK;
}

gw_status gw_mlp_destroy(gw_mlp *m)
{
    if (!m)
        return GW_OK;
    cudaSetDevice(m->device);
    if (m->stream)
        cudaStreamSynchronize(m->stream);
    else
        cudaDeviceSynchronize();
    void *ptrs[] = {m->theta, m->grad,   m->m,      m->v,      m->theta16, m->w32,  m->H[0],  m->H[1],
                    m->H[2],  m->Da,     m->Db,     m->D4,     m->Y,       m->part, m->pX,    m->pXc,
                    m->pH[0], m->pH[1],  m->pHc[0], m->pHc[1], m->pD[0],   m->pD[1], m->pDc,  m->pW[0], m->pW[1],
                    m->pW[2], m->pWc[0], m->pWc[1], m->csum,   m->Wt,      m->d_err};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    cudaGetLastError();
    delete m;
    return GW_OK;
}

gw_status gw_mlp_last_error(gw_mlp *m, char *buf, size_t len)
{
    if (!m || !buf || !len)
        return GW_E_INVALID;
    snprintf(buf, len, "%s", m->last_error.c_str());
    return GW_OK;
}

gw_status gw_mlp_set_params(gw_mlp *m, const float *theta, int on_device)
{
    MLP_TRY(check_mlp(m));
    if (!theta)
        return mfail(m, GW_E_INVALID, "gw_mlp_set_params: null parameter pointer");
    const size_t bytes = (size_t)m->P * sizeof(float);
    MLP_CUDA(cudaMemcpyAsync(m->theta, theta, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             m->stream),
             "gw_mlp_set_params copy");
    MLP_CUDA(cudaMemsetAsync(m->m, 0, bytes, m->stream), "gw_mlp_set_params reset");
    MLP_CUDA(cudaMemsetAsync(m->v, 0, bytes, m->stream), "gw_mlp_set_params reset");
    to_half_kernel<<<(int)std::min<long>((m->P + 255) / 256, 4L * m->num_sms), 256, 0, m->stream>>>(
        m->theta, m->theta16, m->w32, m->P);
    gw::count_launches(1);
    MLP_CUDA(cudaGetLastError(), "gw_mlp_set_params convert");
    m->step = 0;
    m->tiled = false;
    m->wpacked = false;
    if (!on_device)
        MLP_CUDA(cudaStreamSynchronize(m->stream), "gw_mlp_set_params sync");
    return GW_OK;
}

gw_status gw_mlp_get_params(gw_mlp *m, float *theta, int on_device)
{
    MLP_TRY(check_mlp(m));
    if (!theta)
        return mfail(m, GW_E_INVALID, "gw_mlp_get_params: null parameter pointer");
    MLP_CUDA(cudaMemcpyAsync(theta, m->theta, (size_t)m->P * sizeof(float),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream),
             "gw_mlp_get_params copy");
    if (!on_device)
        MLP_CUDA(cudaStreamSynchronize(m->stream), "gw_mlp_get_params sync");
    return GW_OK;
}

gw_status gw_mlp_forward(gw_mlp *m, const float *X, long n, float *Y)
{
    MLP_TRY(check_mlp(m));
    if (!X || !Y || n < 0)
        return mfail(m, GW_E_INVALID, "gw_mlp_forward: null pointer or negative size");
    for (long b0 = 0; b0 < n; b0 += m->max_batch) {
        const int b = (int)std::min<long>(m->max_batch, n - b0);
        MLP_CUDA(forward_batch(m, X + b0 * m->n_in, nullptr, b, Y + b0 * NOUT, false), "gw_mlp_forward");
    }
    return GW_OK;
}

gw_status gw_mlp_infer(gw_mlp *m, const float *X, long n, float *Y)
{
    MLP_TRY(check_mlp(m));
    if (!X || !Y || n < 0)
        return mfail(m, GW_E_INVALID, "gw_mlp_infer: null pointer or negative size");
    if (m->hidden != 256 || m->n_in > 16)
        return mfail(m, GW_E_UNSUPPORTED, "gw_mlp_infer: the tensor-core path takes hidden = 256 and n_in <= 16");
    if (n == 0)
        return GW_OK;
    if (!m->Wt)
        MLP_CUDA(cudaMalloc(&m->Wt, gw::mlp_tc_weights_bytes()), "gw_mlp_infer weights");
    if (!m->tiled) {
        MLP_CUDA(gw::launch_mlp_tile_weights(m->theta16 + m->off_w[0], m->n_in, m->theta16 + m->off_w[1],
                                             m->theta16 + m->off_w[2], m->Wt, m->stream),
                 "gw_mlp_infer tile weights");
        m->tiled = true;
    }
    const uint64_t wait_ns = 2000000000ull;
    MLP_CUDA(gw::launch_mlp_tc_forward(X, n, m->n_in, m->Wt, m->theta + m->off_b[0], m->theta + m->off_b[1],
                                       m->theta + m->off_b[2], m->theta16 + m->off_w[3], m->theta + m->off_b[3], Y,
                                       m->num_sms, m->d_err, wait_ns, m->stream),
             "gw_mlp_infer");
    return GW_OK;
}

gw_status gw_mlp_check(gw_mlp *m)
{
    MLP_TRY(check_mlp(m));
    MLP_CUDA(cudaStreamSynchronize(m->stream), "gw_mlp_check sync");
    if (!m->d_err)
        return GW_OK;
    uint32_t word = 0;
    MLP_CUDA(cudaMemcpy(&word, m->d_err, sizeof word, cudaMemcpyDeviceToHost), "gw_mlp_check readback");
    if (word == 0)
        return GW_OK;
    cudaMemset(m->d_err, 0, sizeof(uint32_t));
    return mfail(m, static_cast<gw_status>(word & 0xFF), "a tensor-core kernel's device-side wait ran out (code %u)",
                 word & 0xFF);
}

gw_status gw_mlp_grad(gw_mlp *m, const float *X, const float *T, const int *rows, int batch, float *grad, float *loss)
{
    MLP_TRY(check_mlp(m));
    if (!X || !T || !grad || !loss || batch < 1 || batch > m->max_batch)
        return mfail(m, GW_E_INVALID, "gw_mlp_grad: null pointer or batch outside [1, max_batch]");
    MLP_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), m->stream), "gw_mlp_grad loss reset");
    MLP_CUDA(loss_grad(m, X, T, rows, batch, loss), "gw_mlp_grad");
    MLP_CUDA(cudaMemcpyAsync(grad, m->grad, (size_t)m->P * sizeof(float), cudaMemcpyDeviceToDevice, m->stream),
             "gw_mlp_grad copy");
    return GW_OK;
}

gw_status gw_mlp_train_step(gw_mlp *m, const float *X, const float *T, const int *rows, int batch, double lr,
                            double beta1, double beta2, double adam_eps, float *loss_accum)
{
    MLP_TRY(check_mlp(m));
    if (!X || !T || batch < 1 || batch > m->max_batch)
        return mfail(m, GW_E_INVALID, "gw_mlp_train_step: null pointer or batch outside [1, max_batch]");
    if (!(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(adam_eps >= 0))
        return mfail(m, GW_E_INVALID, "gw_mlp_train_step: bad optimiser constants");
    return train_step(m, X, T, rows, batch, lr, beta1, beta2, adam_eps, loss_accum);
}

gw_status gw_corr_train(gw_mlp *m, const float *X, const float *T, long n, const gw_corr_train_opts *o,
                        float *losses)
{
    MLP_TRY(check_mlp(m));
    if (!X || !T || !o || !losses || n < 1 || n > 0x7FFFFFFFL)
        return mfail(m, GW_E_INVALID, "gw_corr_train: null pointer or n outside [1, 2^31)");
    if (o->epochs < 1 || o->batch < 1 || o->batch > m->max_batch || o->diag_repeat < 1 ||
        o->diag_feature >= m->n_in)
        return mfail(m, GW_E_INVALID, "gw_corr_train: epochs, batch, diag_repeat or diag_feature out of range");
    if (!(o->lr > 0) || !(o->lr_final >= 0) || !(o->beta1 >= 0 && o->beta1 < 1) || !(o->beta2 >= 0 && o->beta2 < 1) ||
        !(o->adam_eps >= 0))
        return mfail(m, GW_E_INVALID, "gw_corr_train: bad optimiser constants");
    MLP_CUDA(cudaSetDevice(m->device), "gw_corr_train device");
    cudaStream_t s = m->stream;
    // device scratch of this call: the pool and its sorted copy, the sort keys, the diagonal rows
    int *idx = nullptr, *D = nullptr, *pool = nullptr, *order = nullptr, *nd_d = nullptr;
    unsigned char *flags = nullptr;
    unsigned long long *keys = nullptr, *keys_sorted = nullptr;
    float *acc = nullptr;
    void *tmp = nullptr;
    gw_status st = GW_OK;
    auto release = [&]() {
        cudaFree(idx);
        cudaFree(D);
        cudaFree(pool);
        cudaFree(order);
        cudaFree(nd_d);
        cudaFree(flags);
        cudaFree(keys);
        cudaFree(keys_sorted);
        cudaFree(acc);
        cudaFree(tmp);
    };
#define TRAIN_CUDA(call, where)                  \
    do {                                         \
        cudaError_t e_ = (call);                 \
        if (e_ != cudaSuccess) {                 \
            st = mcuda(m, e_, where);            \
            release();                           \
            return st;                           \
        }                                        \
    } while (0)
    // diagonal rows (feature diag_feature set), ascending
    int nd = 0;
    if (o->diag_repeat > 1 && o->diag_feature >= 0) {
        size_t tb = 0;
        TRAIN_CUDA(cudaMalloc(&idx, n * sizeof(int)), "gw_corr_train rows");
        TRAIN_CUDA(cudaMalloc(&D, n * sizeof(int)), "gw_corr_train diagonal rows");
        TRAIN_CUDA(cudaMalloc(&flags, n), "gw_corr_train flags");
        TRAIN_CUDA(cudaMalloc(&nd_d, sizeof(int)), "gw_corr_train count");
        diag_flags_kernel<<<blocks_for(n, m->num_sms), 256, 0, s>>>(X, n, m->n_in, o->diag_feature, flags, idx);
        gw::count_launches(1);
        TRAIN_CUDA(cub::DeviceSelect::Flagged(nullptr, tb, idx, flags, D, nd_d, (int)n, s), "gw_corr_train select");
        TRAIN_CUDA(cudaMalloc(&tmp, tb), "gw_corr_train select scratch");
        TRAIN_CUDA(cub::DeviceSelect::Flagged(tmp, tb, idx, flags, D, nd_d, (int)n, s), "gw_corr_train select");
        TRAIN_CUDA(cudaMemcpyAsync(&nd, nd_d, sizeof(int), cudaMemcpyDeviceToHost, s), "gw_corr_train count");
        TRAIN_CUDA(cudaStreamSynchronize(s), "gw_corr_train count");
        cudaFree(tmp);
        tmp = nullptr;
    }
    const long S = n + (long)(nd > 0 ? o->diag_repeat - 1 : 0) * nd;
    if (S > 0x7FFFFFFFL) {
        release();
        return mfail(m, GW_E_INVALID, "gw_corr_train: pool of %ld rows exceeds 2^31", S);
    }
    const long steps = S / o->batch;
    if (steps < 1) {
        release();
        return mfail(m, GW_E_INVALID, "gw_corr_train: fewer rows than one minibatch");
    }
    size_t sb = 0;
    TRAIN_CUDA(cudaMalloc(&pool, S * sizeof(int)), "gw_corr_train pool");
    TRAIN_CUDA(cudaMalloc(&order, S * sizeof(int)), "gw_corr_train order");
    TRAIN_CUDA(cudaMalloc(&keys, S * sizeof(unsigned long long)), "gw_corr_train keys");
    TRAIN_CUDA(cudaMalloc(&keys_sorted, S * sizeof(unsigned long long)), "gw_corr_train keys");
    TRAIN_CUDA(cudaMalloc(&acc, (size_t)o->epochs * sizeof(float)), "gw_corr_train losses");
    TRAIN_CUDA(cudaMemsetAsync(acc, 0, (size_t)o->epochs * sizeof(float), s), "gw_corr_train losses");
    pool_kernel<<<blocks_for(S, m->num_sms), 256, 0, s>>>(n, D, nd, S, pool);
    gw::count_launches(1);
    TRAIN_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, sb, keys, keys_sorted, pool, order, (int)S, 0, 64, s),
               "gw_corr_train sort");
    TRAIN_CUDA(cudaMalloc(&tmp, sb), "gw_corr_train sort scratch");
    const long total = (long)o->epochs * steps;
    long t = 0;
    for (int e = 0; e < o->epochs; ++e) {
        order_keys_kernel<<<blocks_for(S, m->num_sms), 256, 0, s>>>(o->seed, e, S, keys);
        gw::count_launches(1);
        TRAIN_CUDA(cub::DeviceRadixSort::SortPairs(tmp, sb, keys, keys_sorted, pool, order, (int)S, 0, 64, s),
                   "gw_corr_train sort");
        for (long i = 0; i < steps; ++i, ++t) {
            const double lr_t = o->lr_final + 0.5 * (o->lr - o->lr_final) * (1.0 + std::cos(M_PI * (double)t / total));
            st = train_step(m, X, T, order + i * o->batch, o->batch, lr_t, o->beta1, o->beta2, o->adam_eps, acc + e);
            if (st != GW_OK) {
                release();
                return st;
            }
        }
    }
    std::vector<float> h(o->epochs);
    TRAIN_CUDA(cudaMemcpyAsync(h.data(), acc, h.size() * sizeof(float), cudaMemcpyDeviceToHost, s), "gw_corr_train losses");
    TRAIN_CUDA(cudaStreamSynchronize(s), "gw_corr_train sync");
#undef TRAIN_CUDA
    for (int e = 0; e < o->epochs; ++e)
        losses[e] = h[e] / (float)steps;
    release();
    return gw_mlp_check(m);  // the tensor-core kernels' status word
}

gw_status gw_corr_weight_ratio(const double *E_eV, int nv, int nc_keep, int nc_all, float *ratio, void *stream)
{
    if (!E_eV || !ratio || nv < 1 || nv > RATIO_MAX_NV || nc_keep < 1 || nc_all <= nc_keep)
        return GW_E_INVALID;
    weight_ratio_kernel<<<RATIO_CLUSTER, RATIO_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(E_eV, nv, nc_keep,
                                                                                               nc_all, ratio);
    gw::count_launches(1);
    return cudaGetLastError() == cudaSuccess ? GW_OK : GW_E_CUDA;
}

gw_status gw_corr_features(const void *PG, int ng, const int *gvec, int gcut, const float *ratio, const void *PG_clos,
                           float *X, float *scale, void *stream)
{
    if (!PG || !gvec || !ratio || !X || !scale || ng < 2 || gcut < 1)
        return GW_E_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float2 *P = static_cast<const float2 *>(PG);
    entry_scale_kernel<<<1, 256, 0, s>>>(P, ng, scale);
    features_kernel<<<ng, 128, 0, s>>>(P, ng, gvec, 1.f / (float)gcut, ratio, static_cast<const float2 *>(PG_clos),
                                       scale, X);
    gw::count_launches(2);
    return cudaGetLastError() == cudaSuccess ? GW_OK : GW_E_CUDA;
}

gw_status gw_corr_targets(const void *PG_lo, const void *PG_hi, const void *PG_clos, int ng, const float *scale,
                          float *T, void *stream)
{
    if (!PG_lo || !PG_hi || !scale || !T || ng < 1)
        return GW_E_INVALID;
    targets_kernel<<<ng, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const float2 *>(PG_lo), static_cast<const float2 *>(PG_hi), static_cast<const float2 *>(PG_clos),
        ng, scale, T);
    gw::count_launches(1);
    return cudaGetLastError() == cudaSuccess ? GW_OK : GW_E_CUDA;
}

gw_status gw_corr_apply(void *PG, int ng, const float *Y, const float *scale, const void *PG_clos, void *stream)
{
    if (!PG || !Y || !scale || ng < 1)
        return GW_E_INVALID;
    apply_kernel<<<ng, 128, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<float2 *>(PG), ng, Y, scale,
                                                                      static_cast<const float2 *>(PG_clos));
    gw::count_launches(1);
    return cudaGetLastError() == cudaSuccess ? GW_OK : GW_E_CUDA;
}

}  // extern "C"
