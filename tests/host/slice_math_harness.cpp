// CPU run of the per-trace slice arithmetic of csrc/slice_math.cuh.
// Reads lines "A B k Lq W" (A, B unsigned 64-bit) from stdin and prints
// "u0 z0 ph phi_0 ... phi_{W-1}" with beta = 2.3 W; the test compares them
// with exact integer arithmetic and the kernel formula in numpy.
#include <cstdio>
#include <cstdlib>

#include "../../paper_2505_00387_gb300/csrc/slice_math.cuh"

using namespace aahrt;

template <int W>
static void run(unsigned long long A, unsigned long long B, unsigned k, int Lq) {
    const TapSet t = trace_taps<W>(A, B, k, Lq);
    float phi[W];
    es_weights<W>(t.z0, 2.3f * W, phi);
    printf("%d %.9g %.9g", t.u0, t.z0, t.ph);
    for (int i = 0; i < W; ++i) printf(" %.9g", phi[i]);
    printf("\n");
}

int main() {
    unsigned long long A, B;
    unsigned k;
    int Lq, W;
    while (scanf("%llu %llu %u %d %d", &A, &B, &k, &Lq, &W) == 5) {
        switch (W) {
            case 4: run<4>(A, B, k, Lq); break;
            case 5: run<5>(A, B, k, Lq); break;
            case 6: run<6>(A, B, k, Lq); break;
            case 7: run<7>(A, B, k, Lq); break;
            case 8: run<8>(A, B, k, Lq); break;
            default: printf("bad W\n"); return 1;
        }
    }
    return 0;
}
