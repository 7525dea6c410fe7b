// CPU check of the shared-memory FFT groups of csrc/fft.cuh: the same
// dif_group / dit_group code, driven sequentially on the host, against an
// explicit O(N^2) DFT in double precision.  Prints the worst relative error
// per length and transform kind; exit status 1 when any exceeds 1e-5.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_2505_00387_gb300/csrc/fft.cuh"

using namespace aahrt;

static std::vector<float2> twiddles(int L) {
    const int N = 1 << L;
    std::vector<float2> tw(N / 2 > 0 ? N / 2 : 1);
    for (int m = 0; m < N / 2; ++m) {
        const double a = -2.0 * M_PI * m / N;
        tw[m] = make_float2((float)cos(a), (float)sin(a));
    }
    return tw;
}

int main() {
    srand(1234);
    double worst_all = 0.0;
    for (int L = 1; L <= 13; ++L) {
        const int N = 1 << L;
        std::vector<float2> tw = twiddles(L);
        std::vector<double> xr(N), xi(N);
        for (int n = 0; n < N; ++n) {
            xr[n] = rand() / (double)RAND_MAX - 0.5;
            xi[n] = rand() / (double)RAND_MAX - 0.5;
        }
        double worst[4] = {0, 0, 0, 0};
        for (int kind = 0; kind < 4; ++kind) {
            const bool inv = kind & 1;      // sign +
            const bool dit = kind & 2;      // bit-reversed in, natural out
            std::vector<float2> buf(padded_len(N));
            for (int n = 0; n < N; ++n) {
                const int pos = dit ? (int)brev_bits(n, L) : n;
                buf[padi(pos)] = make_float2((float)xr[n], (float)xi[n]);
            }
            if (!dit && !inv) host_fft<true, false>(buf.data(), L, tw.data());
            if (!dit && inv) host_fft<true, true>(buf.data(), L, tw.data());
            if (dit && !inv) host_fft<false, false>(buf.data(), L, tw.data());
            if (dit && inv) host_fft<false, true>(buf.data(), L, tw.data());
            double num = 0, den = 0;
            for (int k = 0; k < N; ++k) {
                double sr = 0, si = 0;
                const double sg = inv ? 2.0 : -2.0;
                for (int n = 0; n < N; ++n) {
                    const double a = sg * M_PI * (double)((long long)k * n % N) / N;
                    sr += xr[n] * cos(a) - xi[n] * sin(a);
                    si += xr[n] * sin(a) + xi[n] * cos(a);
                }
                const int pos = dit ? k : (int)brev_bits(k, L);
                const float2 g = buf[padi(pos)];
                num += (g.x - sr) * (g.x - sr) + (g.y - si) * (g.y - si);
                den += sr * sr + si * si;
            }
            worst[kind] = sqrt(num / den);
            if (worst[kind] > worst_all) worst_all = worst[kind];
        }
        printf("N=%5d  dif_fwd %.2e  dif_inv %.2e  dit_fwd %.2e  dit_inv %.2e\n", N,
               worst[0], worst[1], worst[2], worst[3]);
    }
    printf("worst %.3e\n", worst_all);
    return worst_all < 1e-5 ? 0 : 1;
}
