// Compile-time twiddles of the constant-twiddle sphere transforms (k_dft.cu): cos(2 pi q / n) and
// sin(2 pi q / n) from the Taylor series of cosine and sine after an exact integer reduction of the
// angle to [0, pi/4], evaluated in FP64 (by the compiler, where they initialise a constant) and
// rounded to FP32 once.  Plain C++17, so a host program compiles the same functions to check every
// constant the kernels use against correctly rounded values.
#pragma once

namespace gw {
namespace twiddle {

constexpr double kPi = 3.14159265358979323846;

constexpr double taylor_cos(double x)  // |x| <= pi/4: 12 terms leave < 1e-28
{
    double term = 1.0, sum = 1.0;
    for (int k = 1; k <= 12; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}

constexpr double taylor_sin(double x)  // |x| <= pi/4
{
    double term = x, sum = x;
    for (int k = 1; k <= 12; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}

// cos(2 pi q / n): r = q mod n folded to [0, n/2] (cosine is even about pi); the angle is then
// (pi/2) u / n with u = 4 r, folded to u <= n by cos(pi - t) = -cos t, and above pi/4 taken as
// sin(pi/2 - t).
constexpr double cos_turn(long long q, long long n)
{
    long long r = q % n;
    if (r < 0)
        r += n;
    if (2 * r > n)
        r = n - r;
    long long u = 4 * r;
    double sg = 1.0;
    if (u > n) {
        u = 2 * n - u;
        sg = -1.0;
    }
    if (2 * u > n)
        return sg * taylor_sin(0.5 * kPi * (double)(n - u) / (double)n);
    return sg * taylor_cos(0.5 * kPi * (double)u / (double)n);
}

template <int N, int Q>
constexpr float kcos = static_cast<float>(cos_turn(Q, N));
template <int N, int Q>  // sin(2 pi q / n) = cos(2 pi (4 q - n) / (4 n))
constexpr float ksin = static_cast<float>(cos_turn(4LL * Q - N, 4LL * N));

}  // namespace twiddle
}  // namespace gw
