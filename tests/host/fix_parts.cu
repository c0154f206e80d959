// Host harness for fix_parts (fixed_sum.cuh), the split behind fix_add_cvt:
// reads lines "count b1 b2 ..." (the bit patterns of count FP32 values with
// |x| < 16, in hex), adds t 2^50 + l of each value in 128-bit integers and
// prints the sum (hi word, lo word, hex).
#include <cstdio>
#include <cstring>

#include "fixed_sum.cuh"

int main() {
    int count;
    while (std::scanf("%d", &count) == 1) {
        grv::u128 acc = 0;
        for (int i = 0; i < count; ++i) {
            unsigned b;
            if (std::scanf("%x", &b) != 1) return 1;
            float x;
            std::memcpy(&x, &b, 4);
            long long t, l;
            grv::fix_parts(x, t, l);
            acc += (grv::u128)((__int128)t << 50) + (grv::u128)(__int128)l;
        }
        std::printf("%016llx %016llx\n", (unsigned long long)(acc >> 64), (unsigned long long)acc);
    }
    return 0;
}
