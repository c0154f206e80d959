// Host harness for the float-float helpers (phase_ops.cuh): reads lines
// "op ahi alo bhi blo [chi clo dhi dlo]" of float bit patterns in hex and
// prints the result's bits: op 0 = ff_add(a, b), 1 = ff_mul(a, b),
// 2 = cff_mul(a + i b, c + i d) (four words: re hi, re lo, im hi, im lo).
#include <cstdio>
#include <cstring>

#include "phase_ops.cuh"

static float f(unsigned u) {
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}
static unsigned u(float x) {
    unsigned v;
    std::memcpy(&v, &x, 4);
    return v;
}

int main() {
    using namespace grv::ph;
    int op;
    while (std::scanf("%d", &op) == 1) {
        unsigned w[8] = {0};
        const int nw = op == 2 ? 8 : 4;
        for (int i = 0; i < nw; ++i)
            if (std::scanf("%x", &w[i]) != 1) return 1;
        if (op == 0 || op == 1) {
            const ff a{f(w[0]), f(w[1])}, b{f(w[2]), f(w[3])};
            const ff r = op == 0 ? ff_add(a, b) : ff_mul(a, b);
            std::printf("%08x %08x\n", u(r.hi), u(r.lo));
        } else {
            const cff a{ff{f(w[0]), f(w[1])}, ff{f(w[2]), f(w[3])}}, b{ff{f(w[4]), f(w[5])}, ff{f(w[6]), f(w[7])}};
            const cff r = cff_mul(a, b);
            std::printf("%08x %08x %08x %08x\n", u(r.re.hi), u(r.re.lo), u(r.im.hi), u(r.im.lo));
        }
    }
    return 0;
}
