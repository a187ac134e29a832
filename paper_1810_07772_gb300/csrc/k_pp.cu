// The von der Linden-Horsch plasmon-pole model of Sec. 5.2 on top of eps^-1:
//   S = sqrt(V) (eps^-1 - I) sqrt(V), Hermitian and negative semidefinite (eps >= I);
//   its most negative eigenpairs (sigma_a, A_a), Eq. (eigdecomp), by block subspace iteration
//   with Rayleigh-Ritz in FP64;
//   the mode frequencies from the Johnson sum rule, Eq. (ppfreq),
//     omega_a^2 = -(1/sigma_a) A_a^H Omega A_a,
//     Omega_gg' = V(q+g) V(q+g') ((q+g).(q+g')) rho(g - g'),  rho(G) = sum_r e^{-iG.r} 2 sum_v |psi_v(r)|^2;
//   and S(omega) = sum_a A_a sigma_a omega_a^2 / (omega_a^2 - omega^2) A_a^H, Eq. (ppform).
// The dense products go through the FP64 zgemm of k_eps.cu; the b x b steps (Cholesky of the
// Gram matrix, Jacobi of the Rayleigh quotient) run in one CTA (b <= 40).
#include <algorithm>
#include <cmath>
#include <vector>

#include "gw_internal.cuh"

namespace gw {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ double2 cmulc(double2 a, double2 b)  // conj(a) b
{
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// rho(r) = 2 sum_{v < nv} |psi_v(r)|^2 from the transposed states [N_r][nb], as complex (rho, 0).
__global__ void density_kernel(const float2 *__restrict__ psiT, int nr, int nb, int nv, double2 *__restrict__ rho)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int v = 0; v < nv; ++v) {
            const float2 z = psiT[(size_t)r * nb + v];
            s += (double)z.x * z.x + (double)z.y * z.y;
        }
        rho[r] = make_double2(2.0 * s, 0.0);
    }
}

// out[..., m, ...] = sum_j in[..., j, ...] e^{-2 pi i m j / n} along the axis with the given
// stride; tw[t] = e^{-2 pi i t / n} (FP64).
__global__ void dft_axis64_kernel(const double2 *__restrict__ in, double2 *__restrict__ out, int nr, int n, int stride,
                                  const double2 *__restrict__ tw)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        const int m = (r / stride) % n;
        const int base = r - m * stride;
        double2 acc = make_double2(0.0, 0.0);
        int t = 0;
        for (int j = 0; j < n; ++j) {
            const double2 v = in[base + j * stride], w = tw[t];
            acc.x = fma(v.x, w.x, fma(-v.y, w.y, acc.x));
            acc.y = fma(v.x, w.y, fma(v.y, w.x, acc.y));
            t += m;
            if (t >= n)
                t -= n;
        }
        out[r] = acc;
    }
}

// S = sqrt(V) (eps^-1 - I) sqrt(V), Hermitian part.
__global__ void pp_S_kernel(const double2 *__restrict__ inv, const double *__restrict__ sv, int ng,
                            double2 *__restrict__ S)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = blockIdx.y; i < ng && j < ng; i += gridDim.y) {
        const double2 a = inv[(size_t)i * ng + j], b = inv[(size_t)j * ng + i];
        const double d = i == j ? 1.0 : 0.0;
        const double w = sv[i] * sv[j];
        S[(size_t)i * ng + j] = make_double2(w * (0.5 * (a.x + b.x) - d), w * 0.5 * (a.y - b.y));
    }
}

// Omega_ij = V_i V_j (k_i . k_j) rho((m_i - m_j) mod n), V = sv^2, k = (2 pi / L)(m + q).
__global__ void pp_omega_kernel(const int *__restrict__ gvec, const double *__restrict__ sv, int ng, int n1, int n2,
                                int n3, double kx0, double q0, double q1, double q2,
                                const double2 *__restrict__ rhoG, double2 *__restrict__ W)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = blockIdx.y; i < ng && j < ng; i += gridDim.y) {
        const int *mi = gvec + 3 * i, *mj = gvec + 3 * j;
        const double ki0 = kx0 * (mi[0] + q0), ki1 = kx0 * (mi[1] + q1), ki2 = kx0 * (mi[2] + q2);
        const double kj0 = kx0 * (mj[0] + q0), kj1 = kx0 * (mj[1] + q1), kj2 = kx0 * (mj[2] + q2);
        const int d0 = ((mi[0] - mj[0]) % n1 + n1) % n1, d1 = ((mi[1] - mj[1]) % n2 + n2) % n2,
                  d2 = ((mi[2] - mj[2]) % n3 + n3) % n3;
        const double2 rho = rhoG[((size_t)d0 * n2 + d1) * n3 + d2];
        const double f = sv[i] * sv[i] * sv[j] * sv[j] * (ki0 * kj0 + ki1 * kj1 + ki2 * kj2);
        W[(size_t)i * ng + j] = make_double2(f * rho.x, f * rho.y);
    }
}

// Deterministic start block R [ng][b]: splitmix64 of the index, two uniforms in [-1, 1).
__global__ void pp_random_kernel(double2 *__restrict__ R, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        unsigned long long z = (i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double a = (double)(z >> 11) * 0x1.0p-53, b = (double)(z & 0x1FFFFFull) * 0x1.0p-21;
        R[i] = make_double2(2.0 * a - 1.0, 2.0 * b - 1.0);
    }
}

// out[0] = max_i |S_ii| (one block).
__global__ void diag_absmax_kernel(const double2 *__restrict__ S, int ng, double *out)
{
    __shared__ double red[256];
    double m = 0.0;
    for (int i = threadIdx.x; i < ng; i += blockDim.x)
        m = fmax(m, fabs(S[(size_t)i * ng + i].x));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        out[0] = red[0];
}

// Y = c X - Y: the step of the shifted operator c I - S, given Y = S X.
__global__ void shift_step_kernel(const double2 *__restrict__ X, double2 *__restrict__ Y, double c, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 x = X[i], y = Y[i];
        Y[i] = make_double2(c * x.x - y.x, c * x.y - y.y);
    }
}

// out[b][b] = sum over the nparts partial b x b products (fixed order).
__global__ void sum_parts64_kernel(const double2 *__restrict__ parts, int nparts, int n, double2 *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double2 a = parts[i];
        for (int p = 1; p < nparts; ++p) {
            a.x += parts[(size_t)p * n + i].x;
            a.y += parts[(size_t)p * n + i].y;
        }
        out[i] = a;
    }
}

// One CTA: G (b x b Hermitian positive definite, row-major) = L L^H; U = L^-H (upper), so that
// X U has orthonormal columns when G = X^H X.  flag[0] = 1 if a pivot is not positive.
__global__ void chol_inv_small_kernel(const double2 *__restrict__ G, int b, double2 *__restrict__ U, int *flag)
{
    extern __shared__ double2 sm_ci[];  // L and Li, b x (b + 1) each (dynamic: > 48 KB at b = 40)
    const int P = b + 1;
    double2 *Ls = sm_ci, *Lis = sm_ci + b * P;
#define L(i, j) Ls[(i) * P + (j)]
#define Li(i, j) Lis[(i) * P + (j)]
    const int t = threadIdx.x;
    for (int e = t; e < b * b; e += blockDim.x)
        L(e / b, e % b) = G[e];
    __syncthreads();
    for (int k = 0; k < b; ++k) {
        __shared__ double piv;
        if (t == 0) {
            const double d = L(k, k).x;
            if (!(d > 0.0))
                flag[0] = 1;
            piv = d > 0.0 ? sqrt(d) : 1.0;
            L(k, k) = make_double2(piv, 0.0);
        }
        __syncthreads();
        for (int i = k + 1 + t; i < b; i += blockDim.x)
            L(i, k) = make_double2(L(i, k).x / piv, L(i, k).y / piv);
        __syncthreads();
        for (int e = t; e < (b - k - 1) * (b - k - 1); e += blockDim.x) {
            const int i = k + 1 + e / (b - k - 1), j = k + 1 + e % (b - k - 1);
            if (j <= i) {
                const double2 li = L(i, k), lj = L(j, k);  // L(i, j) -= L(i, k) conj(L(j, k))
                L(i, j).x -= li.x * lj.x + li.y * lj.y;
                L(i, j).y -= li.y * lj.x - li.x * lj.y;
            }
        }
        __syncthreads();
    }
    // Li = L^-1 (lower), column by column: forward substitution, one column per thread
    for (int c = t; c < b; c += blockDim.x) {
        for (int i = 0; i < b; ++i) {
            double2 s = make_double2(i == c ? 1.0 : 0.0, 0.0);
            for (int k = c; k < i; ++k) {
                const double2 p = cmul(L(i, k), Li(k, c));
                s.x -= p.x;
                s.y -= p.y;
            }
            const double d = L(i, i).x;
            Li(i, c) = i < c ? make_double2(0.0, 0.0) : make_double2(s.x / d, s.y / d);
        }
    }
    __syncthreads();
    for (int e = t; e < b * b; e += blockDim.x) {  // U = Li^H
        const int i = e / b, j = e % b;
        const double2 v = Li(j, i);
        U[e] = make_double2(v.x, -v.y);
    }
#undef L
#undef Li
}

// One CTA: cyclic Jacobi with round-robin pair order on a b x b Hermitian H (b even, <= 40):
// H = W diag(theta) W^H.  theta ascending and W's columns in that order on exit.
__global__ void jacobi_small_kernel(const double2 *__restrict__ Hin, int b, int max_sweeps, double *__restrict__ theta,
                                    double2 *__restrict__ Wout)
{
    extern __shared__ double2 sm_jb[];  // A and W, b x (b + 1) each (dynamic: > 48 KB at b = 40)
    const int P = b + 1;
    double2 *As = sm_jb, *Ws = sm_jb + b * P;
#define A(i, j) As[(i) * P + (j)]
#define W(i, j) Ws[(i) * P + (j)]
    __shared__ int order[40];
    __shared__ int pp[20], pq[20];
    __shared__ double pc[20];
    __shared__ double2 ps[20];  // s e^{i phi}
    __shared__ double offn, tot;
    __shared__ int perm[40];
    const int t = threadIdx.x;
    for (int e = t; e < b * b; e += blockDim.x) {
        const int i = e / b, j = e % b;
        A(i, j) = Hin[e];
        W(i, j) = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    for (int i = t; i < b; i += blockDim.x)
        order[i] = i;
    __syncthreads();
    const int h = b / 2;
    for (int sw = 0; sw < max_sweeps; ++sw) {
        if (t == 0) {
            double o = 0.0, a = 0.0;
            for (int i = 0; i < b; ++i)
                for (int j = 0; j < b; ++j) {
                    const double m2 = A(i, j).x * A(i, j).x + A(i, j).y * A(i, j).y;
                    a += m2;
                    if (i != j)
                        o += m2;
                }
            offn = o;
            tot = a;
        }
        __syncthreads();
        if (!(offn > 1e-30 * tot))
            break;
        for (int step = 0; step < b - 1; ++step) {
            if (t < h) {  // the rotation of pair t: zero A(p, q)
                int p = order[t], q = order[b - 1 - t];
                if (p > q) {
                    const int x = p;
                    p = q;
                    q = x;
                }
                pp[t] = p;
                pq[t] = q;
                const double2 hpq = A(p, q);
                const double ah = sqrt(hpq.x * hpq.x + hpq.y * hpq.y);
                if (ah < 1e-300) {
                    pc[t] = 1.0;
                    ps[t] = make_double2(0.0, 0.0);
                } else {
                    const double tau = (A(q, q).x - A(p, p).x) / (2.0 * ah);
                    const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    const double c = 1.0 / sqrt(1.0 + tt * tt);
                    pc[t] = c;
                    ps[t] = make_double2(tt * c * hpq.x / ah, tt * c * hpq.y / ah);
                }
            }
            __syncthreads();
            // A <- A J (columns p, q): J_pp = J_qq = c, J_pq = s e^{i phi}, J_qp = -s e^{-i phi}
            for (int e = t; e < h * b; e += blockDim.x) {
                const int k = e / b, i = e % b;
                const int p = pp[k], q = pq[k];
                const double c = pc[k];
                const double2 s = ps[k];
                const double2 ap = A(i, p), aq = A(i, q);
                const double2 sc = make_double2(s.x, -s.y);  // conj(s e^{i phi})
                const double2 t1 = cmul(aq, sc), t2 = cmul(ap, s);
                A(i, p) = make_double2(c * ap.x - t1.x, c * ap.y - t1.y);
                A(i, q) = make_double2(t2.x + c * aq.x, t2.y + c * aq.y);
                const double2 wp = W(i, p), wq = W(i, q);
                const double2 u1 = cmul(wq, sc), u2 = cmul(wp, s);
                W(i, p) = make_double2(c * wp.x - u1.x, c * wp.y - u1.y);
                W(i, q) = make_double2(u2.x + c * wq.x, u2.y + c * wq.y);
            }
            __syncthreads();
            // A <- J^H A (rows p, q)
            for (int e = t; e < h * b; e += blockDim.x) {
                const int k = e / b, j = e % b;
                const int p = pp[k], q = pq[k];
                const double c = pc[k];
                const double2 s = ps[k];
                const double2 ap = A(p, j), aq = A(q, j);
                const double2 t1 = cmul(s, aq);                               // s e^{i phi} A_qj
                const double2 t2 = cmul(make_double2(s.x, -s.y), ap);         // s e^{-i phi} A_pj
                A(p, j) = make_double2(c * ap.x - t1.x, c * ap.y - t1.y);
                A(q, j) = make_double2(t2.x + c * aq.x, t2.y + c * aq.y);
            }
            __syncthreads();
            if (t == 0) {  // round robin: keep order[0], rotate the rest
                const int last = order[b - 1];
                for (int i = b - 1; i > 1; --i)
                    order[i] = order[i - 1];
                order[1] = last;
            }
            __syncthreads();
        }
    }
    if (t == 0) {  // ascending eigenvalues (insertion sort of indices)
        for (int i = 0; i < b; ++i)
            perm[i] = i;
        for (int i = 1; i < b; ++i) {
            const int x = perm[i];
            int j = i - 1;
            while (j >= 0 && A(perm[j], perm[j]).x > A(x, x).x) {
                perm[j + 1] = perm[j];
                --j;
            }
            perm[j + 1] = x;
        }
    }
    __syncthreads();
    for (int i = t; i < b; i += blockDim.x)
        theta[i] = A(perm[i], perm[i]).x;
    for (int e = t; e < b * b; e += blockDim.x) {
        const int i = e / b, j = e % b;
        Wout[e] = W(i, perm[j]);
    }
#undef A
#undef W
}

// res[a] = || Y[:, a] - theta[a] X[:, a] || over the first ncol columns (X, Y [ng][ld]).
__global__ void resid_kernel(const double2 *__restrict__ X, const double2 *__restrict__ Y, int ng, int ld,
                             const double *__restrict__ theta, double *__restrict__ res)
{
    __shared__ double red[256];
    const int a = blockIdx.x;
    double s = 0.0;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
        const double2 y = Y[(size_t)g * ld + a], x = X[(size_t)g * ld + a];
        const double rx = y.x - theta[a] * x.x, ry = y.y - theta[a] * x.y;
        s += rx * rx + ry * ry;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        res[a] = sqrt(red[0]);
}

// omega2[a] = -Re(A[:, a]^H T[:, a]) / theta[a]  (A, T [ng][ld]).
__global__ void pp_freq_kernel(const double2 *__restrict__ A, const double2 *__restrict__ T, int ng, int ld,
                               const double *__restrict__ theta, double *__restrict__ omega2)
{
    __shared__ double red[256];
    const int a = blockIdx.x;
    double s = 0.0;
    for (int g = threadIdx.x; g < ng; g += blockDim.x)
        s += cmulc(A[(size_t)g * ld + a], T[(size_t)g * ld + a]).x;
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        omega2[a] = -red[0] / theta[a];
}

// B[g][a] = A[g][a] f_a with f_a = sigma_a omega_a^2 / (omega_a^2 - w^2), a < nuse.
__global__ void pp_scale_kernel(const double2 *__restrict__ A, int ng, int ld, int nuse, const double *__restrict__ sigma,
                                const double *__restrict__ omega2, double w, double2 *__restrict__ B)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ng * nuse; e += gridDim.x * blockDim.x) {
        const int g = e / nuse, a = e - (e / nuse) * nuse;
        const double f = sigma[a] * omega2[a] / (omega2[a] - w * w);
        const double2 v = A[(size_t)g * ld + a];
        B[e] = make_double2(f * v.x, f * v.y);
    }
}

size_t small_smem(int b)
{
    return (size_t)2 * b * (b + 1) * sizeof(double2);
}

int blocks_for(size_t n)
{
    return static_cast<int>(std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 8)));
}

dim3 grid2(int rows, int cols)
{
    const int gx = std::max(1, (cols + 255) / 256);
    return dim3(gx, std::max(1, std::min(rows, 152 * 8 / gx)));
}

}  // namespace

// ---------------------------------------------------------------------------- host side

PPWork PPWork::carve(void *base, int ng, int b, int nr)
{
    PPWork w{};
    uint8_t *p = static_cast<uint8_t *>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void *r = p ? p + off : nullptr;
        off += (bytes + 255) / 256 * 256;
        return r;
    };
    const size_t nn = (size_t)ng * ng, nb = (size_t)ng * b;
    const int nparts = (ng + 15) / 16;
    w.S = static_cast<double2 *>(take(nn * sizeof(double2)));
    w.Om = static_cast<double2 *>(take(nn * sizeof(double2)));
    w.X = static_cast<double2 *>(take(nb * sizeof(double2)));
    w.Y = static_cast<double2 *>(take(nb * sizeof(double2)));
    w.T = static_cast<double2 *>(take(nb * sizeof(double2)));
    w.G = static_cast<double2 *>(take((size_t)b * b * sizeof(double2)));
    w.U = static_cast<double2 *>(take((size_t)b * b * sizeof(double2)));
    w.parts = static_cast<double2 *>(take((size_t)nparts * b * b * sizeof(double2)));
    w.partsY = static_cast<double2 *>(take((size_t)((ng + 63) / 64) * nb * sizeof(double2)));
    w.theta = static_cast<double *>(take(b * sizeof(double)));
    w.res = static_cast<double *>(take(b * sizeof(double)));
    w.omega2 = static_cast<double *>(take(b * sizeof(double)));
    w.rho = static_cast<double2 *>(take((size_t)nr * sizeof(double2)));
    w.rho2 = static_cast<double2 *>(take((size_t)nr * sizeof(double2)));
    w.tw = static_cast<double2 *>(take(3 * 64 * sizeof(double2)));
    w.gvec = static_cast<int *>(take((size_t)3 * ng * sizeof(int)));
    w.flag = static_cast<int *>(take(64));
    w.bytes = off;
    return w;
}

namespace {

// C (b x b) = X^H Y for X, Y [ng][ld] (first b columns), K split into 16-row parts summed in order.
cudaError_t gram(const double2 *X, const double2 *Y, int ng, int ld, int b, double2 *parts, double2 *C, cudaStream_t s)
{
    const int kc = 16, nparts = (ng + kc - 1) / kc;
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    cudaError_t e = launch_zgemm_batched(b, b, kc, one, X, ld, 1, (long)kc * ld, Y, ld, 0, (long)kc * ld, zero, parts,
                                         b, (long)b * b, nparts - 1, s, 0);
    if (e != cudaSuccess)
        return e;
    const int last = ng - (nparts - 1) * kc;  // the ragged last part
    e = launch_zgemm(b, b, last, one, X + (size_t)(nparts - 1) * kc * ld, ld, 1, Y + (size_t)(nparts - 1) * kc * ld,
                     ld, 0, zero, parts + (size_t)(nparts - 1) * b * b, b, s, 0);
    if (e != cudaSuccess)
        return e;
    sum_parts64_kernel<<<blocks_for((size_t)b * b), 256, 0, s>>>(parts, nparts, b * b, C);
    count_launches(1);
    return cudaGetLastError();
}

// Y (ng x b) = A (ng x ng) X (ng x b): K split into 64-wide parts (a batched product, enough CTAs
// for FP64 on every SM), the parts summed in order.
cudaError_t prod_ksplit(const double2 *A, const double2 *X, int ng, int b, double2 *parts, double2 *Y, cudaStream_t s)
{
    const int kc = 64, nparts = (ng + kc - 1) / kc;
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    cudaError_t e = launch_zgemm_batched(ng, b, kc, one, A, ng, 0, kc, X, b, 0, (long)kc * b, zero, parts, b,
                                         (long)ng * b, nparts - 1, s, 0);
    if (e != cudaSuccess)
        return e;
    const int last = ng - (nparts - 1) * kc;
    e = launch_zgemm(ng, b, last, one, A + (size_t)(nparts - 1) * kc, ng, 0, X + (size_t)(nparts - 1) * kc * b, b, 0,
                     zero, parts + (size_t)(nparts - 1) * ng * b, b, s, 0);
    if (e != cudaSuccess)
        return e;
    sum_parts64_kernel<<<blocks_for((size_t)ng * b), 256, 0, s>>>(parts, nparts, ng * b, Y);
    count_launches(1);
    return cudaGetLastError();
}

// rho_W(r) = sum_{v < nv} w_v |psi_v(r)|^2 (FP64), as complex (rho_W, 0).
__global__ void weighted_density_kernel(const float2 *__restrict__ psiT, int nr, int nb, int nv,
                                        const double *__restrict__ w, double2 *__restrict__ rho)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int v = 0; v < nv; ++v) {
            const float2 z = psiT[(size_t)r * nb + v];
            s += w[v] * ((double)z.x * z.x + (double)z.y * z.y);
        }
        rho[r] = make_double2(s, 0.0);
    }
}

// out(g, h) = rhoG((m_g - m_h) mod n) - Ph(g, h)
__global__ void closure_combine_kernel(const double2 *__restrict__ rhoG, const int *__restrict__ gvec, int ng, int n1,
                                       int n2, int n3, const float2 *__restrict__ Ph, float2 *__restrict__ out)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    for (int g = blockIdx.y; g < ng && h < ng; g += gridDim.y) {
        const int d0 = ((gvec[3 * g] - gvec[3 * h]) % n1 + n1) % n1;
        const int d1 = ((gvec[3 * g + 1] - gvec[3 * h + 1]) % n2 + n2) % n2;
        const int d2 = ((gvec[3 * g + 2] - gvec[3 * h + 2]) % n3 + n3) % n3;
        const double2 rho = rhoG[((size_t)d0 * n2 + d1) * n3 + d2];
        const float2 p = Ph[(size_t)g * ng + h];
        out[(size_t)g * ng + h] = make_float2((float)(rho.x - (double)p.x), (float)(rho.y - (double)p.y));
    }
}

}  // namespace

size_t closure_work_bytes(int nr)
{
    return (size_t)2 * nr * sizeof(double2) + 3 * 64 * sizeof(double2);
}

cudaError_t closure_set_twiddles(const int dims[3], int nr, void *work, cudaStream_t s)
{
    double2 *tw = static_cast<double2 *>(work) + 2 * (size_t)nr;
    if (dims[0] > 64 || dims[1] > 64 || dims[2] > 64)
        return cudaErrorInvalidValue;
    double2 twh[3 * 64];
    for (int a = 0; a < 3; ++a)
        for (int t = 0; t < dims[a]; ++t) {
            const double ph = -6.283185307179586476925 * t / dims[a];
            twh[64 * a + t] = make_double2(std::cos(ph), std::sin(ph));
        }
    const cudaError_t e = cudaMemcpyAsync(tw, twh, sizeof twh, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return e;
    return cudaStreamSynchronize(s);  // twh is a host local; once per grid
}

namespace {

// out[k][g] = Q[k][g] csw[v nb] / sw[k] with v = k / nc: the pair transforms of gw_build_PG carry
// the weight sqrt(2/(E_c - E_v)) of Eq. (fdef); the closure's projector term needs the same
// matrix elements M_vc(G) with the weight sqrt(-W_v / (N_r - n_in)) instead.
__global__ void closure_rescale_kernel(const float2 *__restrict__ Q, int nc, int ng, const float *__restrict__ csw,
                                       int nb, const float *__restrict__ sw, float2 *__restrict__ out, long long n)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / ng);
        const float r = csw[(size_t)(k / nc) * nb] / sw[k];
        const float2 q = Q[e];
        out[e] = make_float2(q.x * r, q.y * r);
    }
}

}  // namespace

cudaError_t launch_closure_rescale(const float2 *Q, int nv, int nc, int ng, const float *csw, int nb, const float *sw,
                                   float2 *out, cudaStream_t s)
{
    const long long n = (long long)nv * nc * ng;
    if (n <= 0)
        return cudaSuccess;
    const int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
    closure_rescale_kernel<<<grid, 256, 0, s>>>(Q, nc, ng, csw, nb, sw, out, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t closure_enqueue(const float2 *psiT, int nr, int nb, int nv, const double *w, const int dims[3],
                            const int *gvec_dev, int ng, const float2 *Ph, float2 *out, void *work, cudaStream_t s)
{
    double2 *rho = static_cast<double2 *>(work), *rho2 = rho + nr, *tw = rho2 + nr;
    const int n1 = dims[0], n2 = dims[1], n3 = dims[2];
    if (n1 > 64 || n2 > 64 || n3 > 64)
        return cudaErrorInvalidValue;
    weighted_density_kernel<<<blocks_for(nr), 256, 0, s>>>(psiT, nr, nb, nv, w, rho);
    dft_axis64_kernel<<<blocks_for(nr), 256, 0, s>>>(rho, rho2, nr, n3, 1, tw + 128);
    dft_axis64_kernel<<<blocks_for(nr), 256, 0, s>>>(rho2, rho, nr, n2, n3, tw + 64);
    dft_axis64_kernel<<<blocks_for(nr), 256, 0, s>>>(rho, rho2, nr, n1, n2 * n3, tw);
    closure_combine_kernel<<<grid2(ng, ng), 256, 0, s>>>(rho2, gvec_dev, ng, n1, n2, n3, Ph, out);
    count_launches(5);
    return cudaGetLastError();
}

cudaError_t pp_prepare(const PPWork &w, const double2 *epsinv, const double *sv, const float2 *psiT, int ng, int nr,
                       int nb, int nv, const int dims[3], const int *gvec_host, double cell_L, const double q[3],
                       cudaStream_t s)
{
    cudaError_t e;
    pp_S_kernel<<<grid2(ng, ng), 256, 0, s>>>(epsinv, sv, ng, w.S);
    density_kernel<<<blocks_for(nr), 256, 0, s>>>(psiT, nr, nb, nv, w.rho);
    count_launches(2);
    // twiddles e^{-2 pi i t / n} per axis (FP64)
    double2 tw[3 * 64];
    for (int a = 0; a < 3; ++a)
        for (int t = 0; t < dims[a]; ++t) {
            const double ph = -6.283185307179586476925 * t / dims[a];
            tw[64 * a + t] = make_double2(std::cos(ph), std::sin(ph));
        }
    if ((e = cudaMemcpyAsync(w.tw, tw, sizeof tw, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(w.gvec, gvec_host, (size_t)3 * ng * sizeof(int), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return e;
    const int n1 = dims[0], n2 = dims[1], n3 = dims[2];
    dft_axis64_kernel<<<blocks_for(nr), 256, 0, s>>>(w.rho, w.rho2, nr, n3, 1, w.tw + 128);
    dft_axis64_kernel<<<blocks_for(nr), 256, 0, s>>>(w.rho2, w.rho, nr, n2, n3, w.tw + 64);
    dft_axis64_kernel<<<blocks_for(nr), 256, 0, s>>>(w.rho, w.rho2, nr, n1, n2 * n3, w.tw);
    pp_omega_kernel<<<grid2(ng, ng), 256, 0, s>>>(w.gvec, sv, ng, n1, n2, n3, 6.283185307179586476925 / cell_L, q[0],
                                                  q[1], q[2], w.rho2, w.Om);
    count_launches(4);
    // the tables above are host locals: finish their copies before returning
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(s);
}

cudaError_t pp_iterate(PPWork &w, int ng, int b, int nmodes, double tol, int max_iter, int *iters_out,
                       cudaStream_t s)
{
    if (b < 2 || b > 40 || (b & 1))
        return cudaErrorInvalidValue;
    cudaError_t ea = cudaFuncSetAttribute(chol_inv_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)small_smem(40));
    if (ea == cudaSuccess)
        ea = cudaFuncSetAttribute(jacobi_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)small_smem(40));
    if (ea != cudaSuccess)
        return ea;
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    cudaError_t e;
    // The block steps use c I - S (c = 1e-3 max |S_ii|): the same eigenvectors, the most negative
    // sigma become its largest eigenvalues, and it has full rank even where S has not (a
    // rank-deficient S would make the Gram matrices of the block singular).
    diag_absmax_kernel<<<1, 256, 0, s>>>(w.S, ng, w.res);
    count_launches(1);
    double smax = 0.0;
    if ((e = cudaMemcpyAsync(&smax, w.res, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return e;
    const double c = smax > 0.0 ? 1e-3 * smax : 1.0;
    const size_t nb = (size_t)ng * b;
    // X0 = (c I - S) R with a deterministic R
    pp_random_kernel<<<blocks_for(nb), 256, 0, s>>>(w.T, nb);
    count_launches(1);
    if ((e = prod_ksplit(w.S, w.T, ng, b, w.partsY, w.X, s)) != cudaSuccess)
        return e;
    shift_step_kernel<<<blocks_for(nb), 256, 0, s>>>(w.T, w.X, c, nb);
    count_launches(1);
    if ((e = cudaMemsetAsync(w.flag, 0, sizeof(int), s)) != cudaSuccess)
        return e;
    std::vector<double> th(b), res(b);
    *iters_out = max_iter;
    for (int it = 0; it < max_iter; ++it) {
        for (int pass = 0; pass < 2; ++pass) {  // Cholesky QR, twice
            if ((e = gram(w.X, w.X, ng, b, b, w.parts, w.G, s)) != cudaSuccess)
                return e;
            chol_inv_small_kernel<<<1, 256, small_smem(b), s>>>(w.G, b, w.U, w.flag);
            count_launches(1);
            if ((e = launch_zgemm(ng, b, b, one, w.X, b, 0, w.U, b, 0, zero, w.T, b, s, 0)) != cudaSuccess)
                return e;
            std::swap(w.X, w.T);
        }
        if ((e = prod_ksplit(w.S, w.X, ng, b, w.partsY, w.Y, s)) != cudaSuccess)
            return e;
        if (it % 4 != 3 && it + 1 < max_iter) {
            shift_step_kernel<<<blocks_for(nb), 256, 0, s>>>(w.X, w.Y, c, nb);  // next block: (c I - S) X
            count_launches(1);
            std::swap(w.X, w.Y);
            continue;
        }
        // Rayleigh-Ritz: H = X^H S X = W diag(theta) W^H; X <- X W, Y <- Y W
        if ((e = gram(w.X, w.Y, ng, b, b, w.parts, w.G, s)) != cudaSuccess)
            return e;
        jacobi_small_kernel<<<1, 256, small_smem(b), s>>>(w.G, b, 30, w.theta, w.U);
        count_launches(1);
        if ((e = launch_zgemm(ng, b, b, one, w.X, b, 0, w.U, b, 0, zero, w.T, b, s, 0)) != cudaSuccess)
            return e;
        std::swap(w.X, w.T);
        if ((e = launch_zgemm(ng, b, b, one, w.Y, b, 0, w.U, b, 0, zero, w.T, b, s, 0)) != cudaSuccess)
            return e;
        std::swap(w.Y, w.T);
        resid_kernel<<<b, 256, 0, s>>>(w.X, w.Y, ng, b, w.theta, w.res);
        count_launches(1);
        if ((e = cudaMemcpyAsync(th.data(), w.theta, b * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(res.data(), w.res, b * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return e;
        bool done = true;
        for (int a = 0; a < nmodes; ++a)
            done = done && res[a] <= tol * std::fabs(th[0]);
        if (done) {
            *iters_out = it + 1;
            break;
        }
        if (it + 1 < max_iter) {
            shift_step_kernel<<<blocks_for(nb), 256, 0, s>>>(w.X, w.Y, c, nb);
            count_launches(1);
            std::swap(w.X, w.Y);
        }
    }
    // frequencies: T = Omega X, omega2 = -Re(x^H T x) / theta
    if ((e = prod_ksplit(w.Om, w.X, ng, b, w.partsY, w.T, s)) != cudaSuccess)
        return e;
    pp_freq_kernel<<<b, 256, 0, s>>>(w.X, w.T, ng, b, w.theta, w.omega2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t pp_eval(const PPWork &w, int ng, int b, int nuse, double omega, double2 *Sout, cudaStream_t s)
{
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    pp_scale_kernel<<<blocks_for((size_t)ng * nuse), 256, 0, s>>>(w.X, ng, b, nuse, w.theta, w.omega2, omega, w.T);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    return launch_zgemm(ng, ng, nuse, one, w.T, nuse, 0, w.X, b, 1, zero, Sout, ng, s, 0);
}

}  // namespace gw
