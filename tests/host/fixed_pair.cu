// Host harness for fix_to_f32_pair (fixed_sum.cuh): reads lines "hi lo s"
// (x = hi * 2^64 + lo, a two's complement 128-bit integer, in hex; s decimal)
// and prints the bits of the float pair (hi, lo) it returns, in hex.
#include <cstdio>

#include "fixed_sum.cuh"

int main() {
    unsigned long long h, l;
    int s;
    while (std::scanf("%llx %llx %d", &h, &l, &s) == 3) {
        const grv::u128 x = ((grv::u128)h << 64) | l;
        const float2 p = grv::fix_to_f32_pair(x, s);
        unsigned a, b;
        __builtin_memcpy(&a, &p.x, 4);
        __builtin_memcpy(&b, &p.y, 4);
        std::printf("%08x %08x\n", a, b);
    }
    return 0;
}
