// Host program of tests/test_twiddles_cpu.py: prints, for every transform size with compile-time
// twiddles, the FP32 constants the kernels take for cos(2 pi q / n) and sin(2 pi q / n), q in
// [0, 2n) (the second period shows the integer reduction), as "n q cos sin" with hex floats.
#include <cstdio>
#include <utility>

#include "twiddle_const.cuh"

template <int N, int Q>
void row()
{
    std::printf("%d %d %a %a\n", N, Q, (double)gw::twiddle::kcos<N, Q>, (double)gw::twiddle::ksin<N, Q>);
}

template <int N, int... Q>
void rows(std::integer_sequence<int, Q...>)
{
    (row<N, Q>(), ...);
}

int main()
{
    rows<12>(std::make_integer_sequence<int, 24>{});
    rows<16>(std::make_integer_sequence<int, 32>{});
    rows<18>(std::make_integer_sequence<int, 36>{});
    rows<20>(std::make_integer_sequence<int, 40>{});
    rows<24>(std::make_integer_sequence<int, 48>{});
    rows<27>(std::make_integer_sequence<int, 54>{});
    return 0;
}
