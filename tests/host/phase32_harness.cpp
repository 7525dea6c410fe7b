// CPU run of the direct sum's 32-bit phase arithmetic of csrc/slice_math.cuh.
// Reads lines "kA kB n" (kA, kB unsigned 64-bit, n signed, |n| <= 2^30) and
// prints the top word phase_top computes and the exact top word of
// kA + n kB (mod 2^64); the test compares them.
#include <cstdio>

#include "../../paper_2505_00387_gb300/csrc/slice_math.cuh"

using namespace aahrt;

int main() {
    unsigned long long kA, kB;
    long long n;
    while (scanf("%llu %llu %lld", &kA, &kB, &n) == 3) {
        const Phase32 p = phase_consts(kA, kB);
        const unsigned np = (unsigned)((unsigned long long)n + 0x80000000ull);
        const unsigned top = phase_top(np, p);
        const unsigned long long exact = kA + (unsigned long long)n * kB;
        printf("%u %u\n", top, (unsigned)(exact >> 32));
    }
    return 0;
}
