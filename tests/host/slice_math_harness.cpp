// CPU run of the per-trace slice arithmetic of csrc/slice_math.cuh.
// Reads lines "A B k Lq W beta" (A, B unsigned 64-bit) from stdin and prints
// "u0 g ph phi_0 ... phi_{W-1}" using the host-fitted kernel polynomial; the
// test compares them with exact integer arithmetic and the kernel formula.
#include <cstdio>
#include <cstdlib>

#include "../../paper_2505_00387_gb300/csrc/slice_math.cuh"

using namespace aahrt;

template <int W>
static void run(unsigned long long A, unsigned long long B, unsigned k, int Lq, double beta) {
    EsPoly P;
    fit_es_poly(W, beta, &P);
    const TapSet t = trace_taps<W>(A, B, k, Lq);
    float phi[W];
    es_weights<W>(P, t.g, phi);
    printf("%d %.9g %.9g", t.u0, t.g, t.ph);
    for (int i = 0; i < W; ++i) printf(" %.9g", phi[i]);
    printf("\n");
}

int main() {
    unsigned long long A, B;
    unsigned k;
    int Lq, W;
    double beta;
    while (scanf("%llu %llu %u %d %d %lf", &A, &B, &k, &Lq, &W, &beta) == 6) {
        switch (W) {
            case 4: run<4>(A, B, k, Lq, beta); break;
            case 5: run<5>(A, B, k, Lq, beta); break;
            case 6: run<6>(A, B, k, Lq, beta); break;
            case 7: run<7>(A, B, k, Lq, beta); break;
            case 8: run<8>(A, B, k, Lq, beta); break;
            case 9: run<9>(A, B, k, Lq, beta); break;
            case 10: run<10>(A, B, k, Lq, beta); break;
            case 11: run<11>(A, B, k, Lq, beta); break;
            case 12: run<12>(A, B, k, Lq, beta); break;
            default: printf("bad W\n"); return 1;
        }
    }
    return 0;
}
